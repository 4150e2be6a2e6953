/*
 * hf.h -- C ABI of the B300 geometric-energy field library.
 *
 * Computes, for two rigid parts given as skeletal densities on a periodic
 * N^3 grid, the geometric energy field over all translations for each
 * sampled rotation of the moving part, together with the force field (its
 * translational gradient) and the torque field (its rotational gradient),
 * and answers pose queries against the precomputed fields.  The method is
 * Behandish & Ilies, "Haptic Assembly Using Skeletal Densities and Fourier
 * Transforms" (ASME JCISE 16(2), 2016):
 *
 *   energy   f(R, t) = integral rho1(p) rho2(R^T (p - t)) dV       Eqs. 1, 3
 *            = F^-1{ F{rho1} . (F{rho2~} o R^T) }                   Eq. 5
 *   force    <df/dt, e> = 2 pi i F^-1{ (e . w) ... }                 Eq. 6a
 *   torque   rotational gradient (the paper's Eq. 6b), here by least
 *            squares over the nearest sampled rotations
 *   query    fields precomputed per permitted orientation, read at a
 *            pose during motion (Section 4.2, "Restricted Motion DOF")
 *
 * Conventions shared by every call:
 *   grid     N^3 nodes on the periodic box [-1,1)^3, spacing h = 2/N, node
 *            index n <-> position -1 + n h, arrays [z][y][x], x fastest,
 *            float32.  Supported N: 32, 64, 96, 128, 256.
 *   lags     field index j <-> translation t = j h (periodic), lag 0 at 0.
 *   E        = +f (the Riemann sum of Eq. 1 with volume element h^3).
 *   F        = -grad_t E (spectral; the Nyquist multiplier on each axis is 0).
 *   T        = -grad_theta E for world-frame perturbations R -> exp([d]x) R,
 *            about the moving part's reference point.
 *   rotation unit quaternion (w, x, y, z); the moving part's density at pose
 *            (R, t) is rho2(R^T (p - t)), sampled by periodic trilinear
 *            interpolation of its grid.
 *
 * Memory: pointers named d_* are device pointers owned by the caller (the
 * library never frees them); h_* are host pointers.  Handles (hf_ctx,
 * hf_part, hf_fieldset, hf_server) are owned by the library, allocated on
 * the context's device and charged against the context's HBM budget; a
 * context must outlive every handle made from it.
 *
 * Streams: every call taking an hf_stream enqueues asynchronous work on it
 * (NULL = the legacy default stream).  Outputs are valid after the stream is
 * synchronised.  A handle produced by a call may be used by later work on
 * the same stream at once.
 *
 * Errors: every call returns an hf_status; no exception or abort crosses the
 * ABI.  On failure the call has written no output handle, and hf_last_error()
 * returns a message for the calling thread.
 *
 * Threads: a context may be shared.  Creating and releasing parts and field
 * sets, computing different field sets, queries and the server's calls are
 * safe from several threads (budget accounting, the profiler and the query
 * mailbox are locked).  One field set must not be computed by two threads at
 * once, nor released while its work runs; hf_autotune / hf_tune_set must not
 * run while field sets of the same context are being created.
 */
#ifndef HF_H
#define HF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HF_OK = 0,
    HF_EINVAL = 1,       /* bad argument (size, pointer, flag, rank-deficient rotation set) */
    HF_ENOMEM = 2,       /* device allocation failed */
    HF_EBUDGET = 3,      /* the allocation would exceed the context's HBM budget */
    HF_ECUDA = 4,        /* a CUDA runtime call failed (message has the CUDA error) */
    HF_ETIMEOUT = 5,     /* a bounded device-side wait gave up */
    HF_ENOTREADY = 6,    /* the field set has not been computed */
    HF_EUNSUPPORTED = 7  /* grid size or flag combination not built */
} hf_status;

typedef struct hf_ctx hf_ctx;
typedef struct hf_part hf_part;
typedef struct hf_fieldset hf_fieldset;
typedef void *hf_stream; /* a cudaStream_t */

/* Part roles for hf_part_create. */
#define HF_STATIONARY 0 /* keeps the scaled half spectrum of rho1 (Section 3.2: precomputed once) */
#define HF_MOVING 1     /* keeps the rho2 grid, resampled per rotation */

/* Field-set flags. */
#define HF_E 0x1u           /* energy field per rotation (always held) */
#define HF_F 0x2u           /* force field (3 components) per rotation (always held) */
#define HF_T 0x4u           /* torque field (3 components) per rotation */
#define HF_TORQUE_F64 0x10u /* torque least-squares product in float64 on the device (over float32 differences) */
/* Torque least-squares product in compensated float32 (Dot2 of Ogita, Rump
 * and Oishi over the float64 operator split into two float32 parts): as
 * accurate as the float64 product before the final rounding to float32, on
 * the float32 units; an alternative to HF_TORQUE_F64 (both: HF_EINVAL). */
#define HF_TORQUE_C 0x200u
/* Precision variant (N = 256 only): the y-axis DFT stages run on the tensor
 * cores as 16 x 16 DFT-matrix GEMMs with operands split into hi + lo parts in
 * BF16 or FP16 and FP32 accumulation; every other stage stays FP32. */
#define HF_PREC_SPLIT_BF16 0x20u
#define HF_PREC_SPLIT_F16 0x40u
/* Spectral mode (Section 3.2, step 1): each rotation's spectrum of the moving
 * part is read off its precomputed spectrum (hf_part_spectral) by trilinear
 * interpolation at R^T omega instead of resampling the grid and transforming
 * it.  The moving part must have a table (HF_ENOTREADY otherwise). */
#define HF_SPECTRAL 0x80u
/* Analytic torque (the rotational gradient of Eq. 6b) in the torque slots
 * instead of the least-squares differences of HF_T: with the moment moved
 * onto the stationary part by integration by parts,
 *   T(t) = C(G, rho2R)(t) - t x F(t),  G(u) = -u x grad rho1(u),
 * C the correlation that gives E, t the signed lag; T = -grad_theta E for
 * world perturbations about the moving part's reference point, exact for the
 * band-limited fields.  Needs hf_part_moments on the stationary part; N <=
 * 128, spatial route (HF_EUNSUPPORTED otherwise); excludes HF_T. */
#define HF_TA 0x100u

/* Field indices for hf_fieldset_get / hf_fieldset_field_ptr and query outputs. */
#define HF_FIELD_E 0
#define HF_FIELD_FX 1
#define HF_FIELD_FY 2
#define HF_FIELD_FZ 3
#define HF_FIELD_TX 4
#define HF_FIELD_TY 5
#define HF_FIELD_TZ 6

/* Library version, e.g. "hf 1.0 sm_103a". Static storage. */
const char *hf_version(void);

/* Thread-local message describing the calling thread's last failure. */
const char *hf_last_error(void);

/* Test hook for the error paths: the nth device, array or pinned-host
 * allocation the library makes from now on (any thread, any handle) fails as
 * if the device were out of memory; nth <= 0 turns it off.  *count (may be
 * NULL) receives the number of allocations made so far, so a test counts an
 * operation's allocations and then fails each in turn.  The allocation-free
 * entry point's own set-up is not counted. */
void hf_inject_alloc_failure(long long nth, long long *count);

/* Create a context on CUDA device `device`.  hbm_budget_bytes bounds the
 * device memory the context's handles may hold (0 = no bound).
 * Errors: HF_EINVAL (null out, bad device), HF_ECUDA. */
hf_status hf_ctx_create(int device, size_t hbm_budget_bytes, hf_ctx **out);
/* Drop the caller's handle.  Every part, field set, batch and server made
 * from the context holds a reference to it, so they may be released before
 * or after this call, in any order; the context's own resources go with the
 * last of them. */
void hf_ctx_destroy(hf_ctx *ctx);
/* Bytes currently charged against the budget, and the budget (0 = none). */
size_t hf_ctx_reserved_bytes(const hf_ctx *ctx);
size_t hf_ctx_budget_bytes(const hf_ctx *ctx);
/* Load now every kernel of the field builds (all grid sizes, launch shapes and
 * precision variants), the torque and the pose queries on the context's
 * device.  CUDA loads device code lazily by default: the first launch of
 * each kernel loads it, and while the driver loads, other threads' launches
 * wait (milliseconds).  A latency-bound caller preloads once at start-up;
 * hf_server_create does.  Loading is per device and idempotent; *loaded (may
 * be NULL) receives the number of kernels in the modules loaded.  The paper
 * has no counterpart: this is the runtime around the method.
 * Errors: HF_EINVAL (null ctx), HF_EUNSUPPORTED (a driver without
 * per-function loading), HF_ECUDA. */
hf_status hf_ctx_preload(hf_ctx *ctx, int *loaded);

/* Skeletal density on the N^3 grid (the stand-in for the paper's skeletal
 * density, Section 2.3): rho[n] = sum_i a_i exp(-|x_n - c_i|^2 / (2 sigma_i^2))
 * over points with |x_n - c_i| <= 6 sigma_i, distances by the minimum image
 * on the period-2 torus.  d_pts: P x 3 (x, y, z); d_sigma: P (> 0, 6 sigma < 1);
 * d_amp: P or NULL (all 1); d_grid_out: N^3, overwritten.  Deterministic.
 * Errors: HF_EINVAL (P < 0, null pointers), HF_EUNSUPPORTED (N), HF_ECUDA. */
hf_status hf_density_build(hf_ctx *ctx, int n, const float *d_pts, const float *d_sigma,
                           const float *d_amp, int P, float *d_grid_out, hf_stream stream);

/* Mesh descriptor (Eq. 2, Section 2.3 "Skeletal Density"; the CAD route of
 * Section 3.1) of a closed triangle mesh with outward orientation on the N^3
 * grid: d_V nv x 3 float64 vertices, d_T nt x 3 int vertex indices (device;
 * checked on the host, HF_EINVAL if out of range).  With eta = |p - q| and
 * xi(p) the signed distance to the surface (negative inside, by the winding
 * number of Eq. 2's inverse-square kernel):
 *   rho(p) = (1/4 pi) integral exp(-(eta/|xi| - 1)^2 / 2 sigma^2) d gamma,
 * d gamma the signed solid-angle element, summed over triangles subdivided
 * 4 ways until each piece subtends at most gamma_max steradians or
 * max_depth (<= 12) is reached.  rho -> the indicator as sigma grows; it is
 * high on the skeleton inside and negative outside.  d_grid_out: N^3 float;
 * d_aux_out (may be NULL): winding number then signed distance, N^3 each.
 * float64 arithmetic; an offline step (every node visits every triangle).
 * Any 2 <= N <= 512 (parts need a supported N).
 * Errors: HF_EINVAL, HF_EUNSUPPORTED, HF_ECUDA. */
hf_status hf_density_mesh(hf_ctx *ctx, int n, const double *d_V, int nv, const int *d_T, int nt, double sigma,
                          double gamma_max, int max_depth, float *d_grid_out, float *d_aux_out,
                          hf_stream stream);

/* Make a part from an N^3 density grid (caller-owned, 8-byte aligned, read by
 * the call's stream work).  HF_STATIONARY parts keep (h^3/N^3) F{rho1} (Eq. 7a with the
 * volume element and the inverse's normalisation folded in); HF_MOVING parts
 * keep a copy of the grid and its support: per axis, the circular range of
 * nodes outside which every slab is zero (a truncated splat leaves most of
 * a padded grid at exactly zero).  The rotated resample reads no texels for
 * samples whose cell lies outside that support on some axis: the cell's
 * corners are zero, so the sample is +0 either way, bit for bit.  With the
 * environment variable HF_SUPPORT=0 at creation the part keeps no support
 * and every sample reads the texture.
 * Errors: HF_EINVAL, HF_EBUDGET, HF_ENOMEM, HF_ECUDA. */
hf_status hf_part_create(hf_ctx *ctx, int n, const float *d_grid, int role, hf_part **out,
                         hf_stream stream);
/* Drops the caller's handle.  Server sessions, their builds in flight and
 * batches hold references of their own: the part's memory is freed when the
 * last of them goes, so the caller may release a part they still use. */
void hf_part_release(hf_part *part);
/* Grid size of a part (0 for NULL). */
int hf_part_n(const hf_part *part);

/* Re-derive a part's stored representation from a new N^3 grid of the same
 * size, in place (no allocation beyond the stream-ordered pool).
 * Errors: HF_EINVAL, HF_ECUDA. */
hf_status hf_part_update(hf_part *part, const float *d_grid, hf_stream stream);

/* Spectral table of a moving part (rotation in the frequency domain,
 * Section 3.2): rho2 zero-padded to os*N nodes per axis (os = 1 or 2, same
 * spacing, the part at the centre), transformed, its phase taken about the
 * physical origin ((-1)^(kx+ky+kz)), kept as a full (os N)^3 complex cube
 * (8 (os N)^3 bytes, charged to the budget; os N must be a supported size).
 * Field sets with HF_SPECTRAL then read the rotated spectrum at frequency
 * k as (-1)^(kx+ky+kz) trilinear_periodic(table, os R^T k~), 0 on every
 * axis's Nyquist plane.  hf_part_update refreshes the table.  Padding (os = 2)
 * halves the frequency step and with it the interpolation error.
 * Errors: HF_EINVAL (not a moving part, os), HF_EUNSUPPORTED, HF_EBUDGET,
 * HF_ENOMEM, HF_ECUDA. */
hf_status hf_part_spectral(hf_part *part, int os, hf_stream stream);
/* The part's table padding factor (0 without a table). */
int hf_part_spectral_os(const hf_part *part);

/* Moment spectra of a stationary part for HF_TA field sets: the spectra of
 * G_a = -(u x grad rho1)_a (u the node position, grad the spectral
 * derivative of the force), 3 half spectra (charged to the budget);
 * hf_part_update refreshes them.  Errors: HF_EINVAL (not stationary),
 * HF_EUNSUPPORTED (N > 128), HF_EBUDGET, HF_ENOMEM, HF_ECUDA. */
hf_status hf_part_moments(hf_part *part, hf_stream stream);

/* Allocate a field set for R rotations at grid size n holding the fields
 * selected by `flags` (energy and force always; HF_T adds torque; at most one
 * of HF_PREC_SPLIT_BF16 / HF_PREC_SPLIT_F16, N = 256 only, else
 * HF_EUNSUPPORTED).  Bytes: R * N^3 * 4 * (#fields) plus per-set scratch.
 * Errors: HF_EINVAL, HF_EBUDGET, HF_ENOMEM, HF_EUNSUPPORTED. */
hf_status hf_fieldset_create(hf_ctx *ctx, int n, int R, unsigned flags, hf_fieldset **out);

/* Compute the fields of `fs` for the rotations h_quat (R x 4, w x y z, host,
 * normalised by the library) of the moving part s2 against the stationary
 * part s1 (Eqs. 3, 5, 6a per rotation; the torque by least squares over the
 * 6 nearest rotations of the set).  R must equal the set's size; with HF_T,
 * R >= 7.  Rotations whose neighbourhood is rank deficient get NaN torque and
 * the call returns HF_EINVAL after enqueueing everything else.  The host
 * preparation of the rotation set (matrices, neighbours, least-squares
 * operators) is kept in `fs` and reused by the next call whose h_quat holds
 * the same bytes; the uploads happen on every call.
 * Errors: HF_EINVAL, HF_ECUDA. */
hf_status hf_fieldset_compute(hf_ctx *ctx, const hf_part *s1, const hf_part *s2,
                              const float *h_quat, int R, hf_fieldset *fs, hf_stream stream);

/* hf_fieldset_create followed by hf_fieldset_compute. */
hf_status hf_fieldset_build(hf_ctx *ctx, const hf_part *s1, const hf_part *s2,
                            const float *h_quat, int R, unsigned flags, hf_fieldset **out,
                            hf_stream stream);

/* Copy field `field` (HF_FIELD_*) of rotation `rot` (N^3 floats) to d_dst.
 * Errors: HF_EINVAL (index out of range or field not held), HF_ENOTREADY, HF_ECUDA. */
hf_status hf_fieldset_get(const hf_fieldset *fs, int rot, int field, float *d_dst, hf_stream stream);

/* Device pointer to field `field` of rotation `rot` inside the set (valid until
 * the set is released).  Errors as hf_fieldset_get. */
hf_status hf_fieldset_field_ptr(const hf_fieldset *fs, int rot, int field, const float **d_ptr);

/* Field-set geometry. */
int hf_fieldset_n(const hf_fieldset *fs);
int hf_fieldset_rotations(const hf_fieldset *fs);
unsigned hf_fieldset_flags(const hf_fieldset *fs);
void hf_fieldset_release(hf_fieldset *fs);

/* Pose query (Section 4.2): the k_blend sampled rotations nearest to q by
 * geodesic angle (ties to the lower index), weights 1/theta normalised (an
 * exact hit, theta < 1e-12, returns that rotation alone); per rotation,
 * periodic trilinear interpolation of each held field at lag u = t/h.
 * out7 = (E, Fx, Fy, Fz, Tx, Ty, Tz); fields not held read 0.  Host in/out;
 * synchronous (runs on an internal high-priority stream, which is not ordered
 * after the stream of hf_fieldset_compute: synchronise that stream first).
 * Errors: HF_EINVAL (k_blend outside 1..8 or > R), HF_ENOTREADY, HF_ECUDA. */
hf_status hf_query(const hf_fieldset *fs, const float t[3], const float q[4], int k_blend,
                   float out7[7]);
/* Answer the context's hf_query calls through the resident query kernel
 * (on != 0) instead of a launch per query, or stop it (on == 0).  A
 * query then posts its request in a mailbox in mapped pinned memory and
 * spins until the kernel, which polls that mailbox, writes the answer back;
 * the answers equal the launched kernel's bit for bit.  An instance of the
 * kernel serves for 10 ms and a context thread keeps the next one queued, so
 * one always runs: meanwhile a device-wide synchronisation (including the
 * one cudaFree implies) waits up to 20 ms.  A query not answered within 20 ms
 * stops the kernel and runs by launch, and so do the context's later queries.
 * On an idle device a launched query is as fast (the launched kernel ranks
 * in float32 first); the resident kernel avoids the launches that builds
 * running beside the queries can hold up for milliseconds.  The paper has
 * no counterpart: this is the runtime around the 1 kHz haptic loop of
 * Section 4.3.  Errors: HF_EINVAL, HF_ECUDA (the kernel did not start). */
hf_status hf_ctx_resident_queries(hf_ctx *ctx, int on);

/* Batched pose query on the caller's stream: d_tq is Q x 7 floats
 * (tx, ty, tz, qw, qx, qy, qz); d_out is Q x 7 floats as in hf_query. */
hf_status hf_query_batch(const hf_fieldset *fs, const float *d_tq, int Q, int k_blend,
                         float *d_out, hf_stream stream);

/* ---- single poses from truncated spectra (the paper's real-time mode) ----
 * Energy, force and torque at an arbitrary pose (R, t), any rotation, from
 * the stationary part's spectrum and the moving part's spectral table
 * (hf_part_spectral), keeping only the modes with |k~_a| <= K on every axis
 * (Section 4.2, "Truncated Inverse FFT"; Section 3.3, low-pass filtering;
 * (2K+1)^3 modes, K = 8 keeps 17^3) and summing the inverse transform at the
 * one translation t instead of over the grid:
 *   S(k) = (h^3/N^3) rho1^(k) conj(B(k)),  B(k) = (-1)^(kx+ky+kz)
 *          trilinear(table, os R^T k~)      (as HF_SPECTRAL field sets)
 *   E = sum Re S e^{i pi k~.t},  F = -grad_t E,  T = -grad_theta E for world
 *   perturbations R -> exp([d]x) R (the exact derivative of the interpolated
 *   sum).  out7 = (E, Fx, Fy, Fz, Tx, Ty, Tz).
 * hf_lowpass_query: host in/out, synchronous (the context's query stream).
 * hf_lowpass_query_batch: d_tq Q x 7 (tx, ty, tz, qw, qx, qy, qz) -> d_out
 * Q x 7 on `stream`.  Errors: HF_EINVAL (parts, K outside 1..N/2-1, bad
 * quaternion), HF_ENOTREADY (no table), HF_ECUDA. */
hf_status hf_lowpass_query(const hf_part *s1, const hf_part *s2, int K, const float t[3], const float q[4],
                           float out7[7]);
hf_status hf_lowpass_query_batch(const hf_part *s1, const hf_part *s2, int K, const float *d_tq, int Q,
                                 float *d_out, hf_stream stream);

/* Device bytes hf_fieldset_create(n, R, flags) charges (0 if unsupported). */
size_t hf_fieldset_bytes(int n, int R, unsigned flags);

/* ---- checkpoints ----
 * Section 3.2 precomputes the parts' densities and spectra before the
 * assembly session and Section 4.2 the fields of the permitted
 * orientations; these save that state to a file and load it back, so that a
 * restarted service does not recompute it.  A file is a concatenation of NPY
 * (version 1.0) arrays, readable one after the other with numpy's
 * np.lib.format.read_array: first an int64 header [tag, version, kind, N,
 * ...], then
 *   kind HF_CKPT_PART: header [.., N, role]; a moving part's grid
 *     (float32 N x N x N, [z][y][x]) or a stationary part's stored spectrum
 *     (complex64 N x N x (N/2+1): (h^3/N^3) DFT(rho1) in the library's
 *     digit-permuted slot order);
 *   kind HF_CKPT_FIELDSET: header [.., N, R, flags, nf, slot[7]]; the
 *     rotations (float32 R x 4, as given to the compute); the fields
 *     (float32 R x nf x N^3, field f of rotation r at slot[f]);
 *   kind HF_CKPT_SESSION (hf_server_session_save): header [.., N, R, flags,
 *     chunks]; the request's rotations (float32 R x 4); the chunk owning each
 *     rotation and its index there (int64 R each); which chunks follow
 *     (int64, one per chunk); then a field-set record (header, rotations,
 *     fields) per resident chunk.
 * Loading reproduces the saved state bit for bit (a moving part's texture
 * and support are rebuilt from its grid).  Saves copy device data through a
 * host buffer on `stream` and return when the file is written; loads
 * allocate as hf_part_create / hf_fieldset_create (charged to the budget)
 * and return with the data on the device.  Errors: HF_EINVAL (open, write,
 * not a checkpoint of this kind, wrong types or shapes), HF_ENOTREADY (a set
 * never computed), HF_EBUDGET, HF_ENOMEM, HF_ECUDA. */
#define HF_CKPT_PART 1
#define HF_CKPT_FIELDSET 2
#define HF_CKPT_SESSION 3
hf_status hf_part_save(const hf_part *p, const char *path, hf_stream stream);
hf_status hf_part_load(hf_ctx *ctx, const char *path, hf_part **out, hf_stream stream);
hf_status hf_fieldset_save(const hf_fieldset *fs, const char *path, hf_stream stream);
hf_status hf_fieldset_load(hf_ctx *ctx, const char *path, hf_fieldset **out, hf_stream stream);
/* Kind, N, R (0 for a part) and flags (a part's role) of a checkpoint file;
 * host only, no GPU. */
hf_status hf_checkpoint_info(const char *path, int *kind, int *n, int *R, unsigned *flags);

/* ---- rotation-set chunking (host only) ----
 * Split R rotations (h_quat R x 4) into chunks whose build sets hold at most
 * max_build rotations, for rotation sets too large for one field set.  A
 * chunk owns a compact group on SO(3): the lowest-index unassigned rotation
 * and its nearest unassigned ones by geodesic angle 2 acos|q_i . q_j|,
 * added while the build set fits.  With halo != 0 the build set is the owned
 * rotations plus the 6 nearest of each in the whole set (the least-squares
 * torque's neighbours, Section 2.4's rotational gradient taken by finite
 * differences), in ascending global index, so an owned rotation's torque
 * from its chunk's set equals the whole set's; max_build must be >= 7.
 * Outputs: h_owner[r] = chunk owning r; chunk c's build set is
 * h_build[h_offsets[c] .. h_offsets[c+1]) (global indices, ascending);
 * h_offsets holds R + 1 ints, h_build build_cap ints (7 R always suffice).
 * Returns the number of chunks, or -1 (bad argument, non-finite quaternion,
 * R < 7 with halo, capacity).  No GPU is used. */
int hf_rotation_chunks(const float *h_quat, int R, int max_build, int halo, int *h_owner, int *h_offsets,
                       int *h_build, int build_cap);

/* ---- serving: sessions, budgeted continuous batching, query lanes ----
 * The restricted-orientation mode of Section 4.2 as a service: sessions keep
 * their parts and their latest field data resident; field-build requests are
 * queued, admitted first-in first-out while the context's HBM budget allows
 * (hf_ctx_create's hbm_budget_bytes), and run concurrently on several build
 * streams, so work admitted mid-flight overlaps on the device.
 *   - A request whose field set exceeds the server's chunk limit (default:
 *     a third of the budget; hf_server_set_chunk_bytes) is split by
 *     hf_rotation_chunks (with torque halos when it asks for HF_T) into
 *     chunks, each its own field set, admitted one by one as memory frees.
 *   - A finished chunk is published at once: a request's first chunk
 *     replaces the session's previous data atomically, later ones fill in.
 *     A session's newer request supersedes its still-queued chunks.
 *   - When nothing runs and the head chunk does not fit, a published chunk
 *     is evicted: the least recently queried of those idle for 20 ms, else
 *     the largest.
 *   - Queries are answered without a kernel launch by a resident query
 *     kernel: the query posts its request in its lane's mailbox in mapped
 *     pinned memory and spins until the kernel writes the answer back.  An
 *     instance of the kernel serves for 10 ms and returns; a server thread
 *     keeps the next instance queued behind it on a high-priority stream, so
 *     one always runs (one SM's worth of warps), and destroying the server
 *     stops it.  A request not answered within 20 ms runs by launch on the
 *     lane's own stream instead.  Since the kernel always runs, a
 *     device-wide synchronisation while a server lives (cudaDeviceSynchronize,
 *     and cudaFree, which implies one) waits for the running and the queued
 *     instance (up to 20 ms).
 *     HF_RESIDENT_QUERIES=0 in the environment makes every query launch.
 *   - Queries run on a pool of high-priority lanes (own stream and pinned
 *     mailbox each) against the chunk that owns the query's nearest rotation
 *     (HF_ENOTREADY if that chunk is not resident); they equal the whole
 *     set's answer when the query's k nearest rotations are owned by it.
 *   - Queries take no lock that the scheduler or a submitting thread holds
 *     (the published data is read through atomic shared pointers).
 *   - At creation the server allocates the context's remaining budget, plus
 *     half again for the gaps between sets of mixed sizes (HF_ARENA_SLACK,
 *     percent; up to the free memory less 4 GB), as one device arena and carves every build's
 *     field set from it with host-side bookkeeping (best fit, coalesced on
 *     free), so that no build maps or unmaps device memory while queries run:
 *     the driver work of a mapping held up other threads' launches for
 *     milliseconds.  A chunk that finds no free range of its size is treated
 *     like one over the budget (eviction, or a wait for a running build).
 *     Without room for the arena the builds allocate from the device's
 *     default stream-ordered pool instead (its reserve kept; trimmed when
 *     the server is destroyed).
 * Request states: 0 queued, 1 running, 2 done, 3 failed, 4 superseded. */
typedef struct hf_server hf_server;
typedef struct {
    int64_t submitted, completed, failed, rejected, superseded, evicted, queries;
    int64_t rotations_completed;
    int queued, running, sessions;
    size_t reserved_bytes, budget_bytes;
    int64_t chunks_submitted, chunks_completed;
    int chunks_resident;
    size_t chunk_bytes;
    /* the device's default memory pool: its reserved bytes now and at their
     * highest (the builds allocate from it only when the server has no arena) */
    size_t pool_reserved_bytes, pool_reserved_high;
    /* the server's field-set arena: its size (0: none), free bytes, largest
     * free range, and the allocations it refused for want of a range */
    size_t arena_bytes, arena_free_bytes, arena_largest_free;
    int64_t arena_refusals;
    /* queries answered by the resident query kernel, those that waited past
     * its bound and ran by launch instead, and whether it is running now */
    int64_t resident_queries, resident_timeouts;
    int resident_live;
} hf_server_stats;

/* max_inflight: builds on the device at once (1..16); query_lanes: 1..64. */
hf_status hf_server_create(hf_ctx *ctx, int max_inflight, int query_lanes, hf_server **out);
void hf_server_destroy(hf_server *srv);
/* Requests whose field set exceeds `bytes` are split into chunks (0: never). */
hf_status hf_server_set_chunk_bytes(hf_server *srv, size_t bytes);
/* A session over a stationary part s1 and a moving part s2 of the same N
 * (the session holds a reference to each until it is closed, and a build of
 * the session in flight holds its own until it completes). */
hf_status hf_server_session_open(hf_server *srv, const hf_part *s1, const hf_part *s2, int *session);
/* Closes a session: its published fields are retired once their readers let
 * go, and its unfinished requests end failed (state 3). */
hf_status hf_server_session_close(hf_server *srv, int session);
/* Queue a field build for R rotations (h_quat R x 4, copied); HF_EBUDGET if
 * it could never fit (unchunked and above the budget, or a chunk of one
 * rotation and its halo above the chunk limit). */
hf_status hf_server_submit(hf_server *srv, int session, const float *h_quat, int R, unsigned flags,
                           int64_t *request);
/* State of a request (0 queued, 1 running, 2 done, 3 failed, 4 superseded)
 * and, once done (every chunk published), its latency submit -> published
 * (ms). */
hf_status hf_server_request_state(hf_server *srv, int64_t request, int *state, double *latency_ms);
/* Number of chunks of a request and (h_owner, R ints, may be NULL) the chunk
 * owning each rotation. */
hf_status hf_server_request_chunks(hf_server *srv, int64_t request, int *chunks, int *h_owner);
/* Pose query against the session's current field data (HF_ENOTREADY if
 * none, or if the chunk owning the nearest rotation is not resident). */
hf_status hf_server_query(hf_server *srv, int session, const float t[3], const float q[4], int k_blend,
                          float out7[7]);
/* Device pointer of field `field` of rotation `rot` (index in the request)
 * of the session's current data (valid while that data stays current). */
hf_status hf_server_field_ptr(hf_server *srv, int session, int rot, int field, const float **d_ptr);
/* Copy that field to d_dst (N^3 floats), on `stream`. */
hf_status hf_server_field_get(hf_server *srv, int session, int rot, int field, float *d_dst, hf_stream stream);
hf_status hf_server_stats_get(hf_server *srv, hf_server_stats *out);
/* A metrics log in JSON lines: appends to `path` one line every period_ms
 * (>= 10) from a thread of its own, and a last line at hf_server_log_close
 * or hf_server_destroy; opening again closes the previous log first.  Each
 * line: t_s (since the server's creation), period_s, the hf_server_stats
 * counters, "query" {n, p50_us, p99_us, p999_us, max_us} of the queries
 * answered in the period, "build" {n, p50_ms, p99_ms, max_ms} of the requests
 * finished in it (submit -> published), and "session_queries" [[session,
 * answered, not_ready], ...] totals of the open sessions.  Percentiles are
 * upper edges of log-spaced bins (8 per octave: within 9%); null when n = 0.
 * Errors: HF_EINVAL (bad period, unopenable path). */
hf_status hf_server_log_open(hf_server *srv, const char *path, int period_ms);
hf_status hf_server_log_close(hf_server *srv);
/* Save a session's published data (its request's rotations and routing and
 * every resident chunk's field set) to a checkpoint file, and restore such a
 * file as the current data of an open session over parts of the same N
 * (typically hf_part_load'ed after a restart); chunks that were not resident
 * stay missing.  Queries and field reads then answer as before the save. */
hf_status hf_server_session_save(hf_server *srv, int session, const char *path);
hf_status hf_server_session_restore(hf_server *srv, int session, const char *path);
/* Queries of a session answered and refused as not ready, so far. */
hf_status hf_server_session_counts(hf_server *srv, int session, int64_t *answered, int64_t *not_ready);
/* Latencies (microseconds, call entry to return) of the queries answered since
 * the last call, oldest first, at most `max` of them (the newest 2^20 are
 * kept); returns how many were written. */
int hf_server_query_latencies(hf_server *srv, float *h_out_us, int max);
/* Diagnostics since the last call, oldest first, 9 doubles per row, at most
 * `max` rows (the newest 4096 are kept); returns the row count.
 *   which 0, queries of 500 us or more: start (ms since hf_server_create),
 *     total us, us spent resolving the session's set, waiting for a lane,
 *     posting the request to the resident query kernel (or, on the launch
 *     path, in the query kernel's launch call), and waiting for the answer
 *     (or in the lane's synchronise); the session; the calling thread's
 *     involuntary and voluntary context switches during the query.
 *   which 1, scheduler calls of 1 ms or more: start (ms), duration (us),
 *     kind (0 field-set create, 1 compute launch, 2 release), then zeros. */
int hf_server_trace(hf_server *srv, int which, double *h_out, int max);
/* Replay pose trajectories against sessions from native threads, one per
 * session, one query every 1/rate_hz seconds (a haptic device's servo loop):
 * h_poses is nsess x steps x 7 (t, q); blocks until every trajectory has run.
 * Latencies go to the latency ring; *answered / *not_ready / *late count the
 * queries answered, refused for want of a field set, and started more than one
 * period late.  Errors: HF_EINVAL. */
hf_status hf_server_drive_queries(hf_server *srv, int nsess, const int *sessions, const float *h_poses, int steps,
                                  double rate_hz, int k_blend, int64_t *answered, int64_t *not_ready,
                                  int64_t *late);

/* Self-check of the bookkeeping behind the server's field-set arena: `ops`
 * seeded random allocations (1 byte to a quarter of the region, log-uniform)
 * and frees on a region of `bytes` at a fictitious address, checking after
 * every step that live ranges are aligned, disjoint and inside the region,
 * that free ranges are coalesced, that a release makes the free range the
 * arena predicted for it, that a free of a freed range is refused,
 * and that a refusal leaves no range with room; at the end everything is
 * freed and the region must be one free range again.  Touches no device
 * memory and needs no GPU.  Returns 0 when every check held, -1 for bad
 * arguments, else the step (1-based; ops + 1 or + 2 for the final checks)
 * that failed.  The paper has no counterpart: this is the server's memory
 * management. */
int64_t hf_arena_selftest(uint64_t seed, size_t bytes, int ops);

/* ---- a scene's precompute as one CUDA graph ----
 * The offline precompute of Section 4.2 for many part pairs at once, each
 * pair with its own grid size (32..256) and its own rotation set: all
 * builds are recorded once into one CUDA graph and replayed with one call.
 * Each pair writes its fields into a slot (a field set).  slots_per_size <= 0
 * gives every pair a slot of its own; slots_per_size = k > 0 lets pairs of
 * the same grid size and rotation count share k slots round-robin, so a
 * scene whose fields exceed the device streams through k sets per size (a
 * slot then holds the last of its pairs after a launch).  Pairs in one slot
 * run in order; slots run concurrently.  The batch holds a reference to each
 * part until it is released.
 *
 *   hf_batch_create      npairs pairs (s1[i] stationary, s2[i] moving, both of
 *                        one size), R[i] rotations each; flags as for
 *                        hf_fieldset_create (HF_T needs R[i] >= 7).
 *                        Errors: HF_EINVAL, HF_EBUDGET, HF_ENOMEM, HF_ECUDA.
 *   hf_batch_set_rotations  pair's R[i] x 4 quaternions (host, copied
 *                        synchronously); may change between launches without
 *                        a new capture, but not while a launch runs.
 *                        HF_EINVAL for a bad quaternion or (after uploading)
 *                        a rank-deficient torque neighbourhood.
 *   hf_batch_capture     record every pair's launches (all pairs need
 *                        rotations; HF_ENOTREADY otherwise) on `lanes`
 *                        concurrent branches (<= 0: one per slot; 1: every
 *                        build in sequence).  Slot s goes to branch s % lanes.
 *                        Make it with no other work of the batch's parts in
 *                        flight; a new capture replaces the previous graph.
 *   hf_batch_launch      enqueue the whole graph on `stream`.
 *   hf_batch_fieldset    the set holding `pair`'s fields after the last
 *                        launch (HF_ENOTREADY if its slot holds another pair);
 *                        the batch owns it: do not release it.
 *   hf_batch_slots       number of slots (field sets) the batch holds. */
typedef struct hf_batch hf_batch;
hf_status hf_batch_create(hf_ctx *ctx, int npairs, const hf_part *const *s1, const hf_part *const *s2,
                          const int *R, unsigned flags, int slots_per_size, hf_batch **out);
hf_status hf_batch_set_rotations(hf_batch *batch, int pair, const float *h_quat);
hf_status hf_batch_capture(hf_batch *batch, int lanes);
/* The batch as ONE launch of a work-queue kernel instead of a graph of
 * per-size kernels (the uneven-batch precompute of Section 4.2 in one
 * launch, recorded as a CUDA graph with the reset of its counters):
 *   - every pair's rotations are cut into chunks of `chunk` rotations (0:
 *     32); each chunk's pass A, B and C blocks are work items, and every
 *     block of the launch takes the next item by ticket from a device
 *     counter, running it with the per-pass kernels' code (256 threads);
 *   - an item waits (bounded, spin_limit polls, 0: about two seconds) only
 *     for items ticketed before it: its pass's producer, and the previous
 *     chunk using its intermediates or its output rotations;
 *   - E and F only, grids 64, 96 and 128; the results equal the per-pass
 *     kernels' bit for bit.
 * self_test bit 0 plants a wait that nothing satisfies, to exercise the
 * bounded wait: hf_batch_status then reports HF_ETIMEOUT, and the context
 * stays usable.  hf_batch_launch runs it.  Errors: HF_EUNSUPPORTED (flags,
 * sizes), HF_ENOTREADY (a pair without rotations), HF_EINVAL, HF_ENOMEM,
 * HF_ECUDA. */
hf_status hf_batch_capture_queue(hf_batch *b, int chunk, long long spin_limit, int self_test);
/* Synchronise `stream` and report the last one-launch run: HF_OK, or
 * HF_ETIMEOUT if a wait ran out; *items and *runs (may be NULL) receive the
 * size of its work queue. */
hf_status hf_batch_status(hf_batch *b, hf_stream stream, int *items, int *runs);
hf_status hf_batch_launch(hf_batch *batch, hf_stream stream);
hf_status hf_batch_fieldset(const hf_batch *batch, int pair, const hf_fieldset **out);
int hf_batch_slots(const hf_batch *batch);
void hf_batch_release(hf_batch *batch);

/* ---- launch-shape autotuning ----
 * Per grid size, the context chooses how many rotations each pass launch
 * covers (the chunk) and whether the slab passes or the pencil pipeline run
 * (N = 256: pencil only).  hf_autotune times builds of E and F on synthetic
 * parts for every candidate that fits the budget, keeps the fastest for field
 * sets created afterwards, and, given a cache_path, first looks for a line
 * for this device and N there (and writes one after timing).  The cache is
 * JSON, one entry per (device, N): chunk, pipeline, pass B and C launch
 * shapes, pipelines, the radix plan, the E+F rate and every timed
 * candidate.  Outputs may be NULL.  hf_tune_set fixes the choice by hand (chunk <= 0 restores the
 * built-in one); hf_tune_get reads the current choice (rot_per_s 0 when not
 * timed).  The environment variable HF_ROT_CHUNK overrides all of them.
 * Errors: HF_EINVAL, HF_EUNSUPPORTED, HF_ENOMEM (nothing fits), HF_ECUDA. */
hf_status hf_autotune(hf_ctx *ctx, int n, const char *cache_path, int *chunk, int *pencil,
                      double *rot_per_s);
hf_status hf_tune_set(hf_ctx *ctx, int n, int chunk, int pencil);
hf_status hf_tune_get(const hf_ctx *ctx, int n, int *chunk, int *pencil, double *rot_per_s);
/* Launch shapes of passes B and C for grid n (the autotuner's compiled
 * candidates, kept in the context like the chunk): tile_b 0 = 32 columns
 * per CTA, 1 = 16; tile_c 0 = the built-in rows per x batch and threads,
 * 1 = 16 rows per x batch, and at N = 128 only 2 = 256 threads per CTA,
 * 3 = that and an L2 prefetch of the block's third input plane, 4 = that
 * and two y-stage items' loads in flight per thread; 5 = each input plane
 * brought into shared memory by bulk copies, the next plane's rows copied as
 * the x transform frees them (256 threads at N = 128), and at N = 128 only
 * 6 = that with 512 threads and 7 = that with the x inverse's digits in the
 * other order (16 x 8: the same fields to rounding, not bit for bit); 5 is
 * the shape used at N = 64, 96, 128 when none was chosen, 0 at other N.
 * Other than 0 only for N = 64, 96, 128.
 * set != 0 stores *tile_b / *tile_c (the
 * fields do not change, only their speed), else reads them.  Errors:
 * HF_EINVAL, HF_EUNSUPPORTED. */
hf_status hf_tune_tiles(hf_ctx *ctx, int n, int set, int *tile_b, int *tile_c);
/* Pipelines a field-set compute at grid n runs (1, or 2 alternating its
 * rotation chunks over two streams so that passes of neighbouring chunks
 * overlap on the device; twice the intermediates).  set != 0 stores *lanes,
 * else reads it.  The HF_LANES environment variable, when set, overrides it;
 * HF_SPECTRAL sets run one pipeline unless that variable says otherwise.
 * Errors: HF_EINVAL, HF_EUNSUPPORTED. */
hf_status hf_tune_lanes(hf_ctx *ctx, int n, int set, int *lanes);

/* Number of tensor-core stage thread blocks whose bounded wait for their own
 * matrix operations gave up since the last reset (each such block wrote no
 * output: the field set computed with it is invalid); -1 if it cannot be read.
 * Synchronous (reads device memory). */
int hf_tc_timeouts(int reset);
/* Number of waits for bulk copies into shared memory (the bulk-staged pass
 * C) that gave up since the last reset; the blocks behind them wrote invalid
 * output.  -1 if it cannot be read.  Synchronous. */
int hf_bulk_timeouts(int reset);
/* Runs one block that bulk-copies 4 KB into shared memory and waits for it
 * with the kernels' bounded wait.  plant = 0: HF_OK if the data arrived and
 * no wait gave up.  plant != 0: the mbarrier expects 16 bytes more than the
 * copy brings, so the wait runs out (about 0.4 s) and counts itself: returns
 * HF_ETIMEOUT with *timeouts the waits that gave up (the context stays
 * usable; reset the counter afterwards).  Errors: HF_EINVAL, HF_ECUDA. */
hf_status hf_bulk_selftest(int device, int plant, int *timeouts);

/* ---- per-kernel timing (CUDA events on the launching stream) ----
 * While enabled, every kernel launch the context's calls make is bracketed by
 * a pair of CUDA events on its stream.  hf_profile_read synchronises the
 * recorded events and accumulates, per kernel kind, the launch count and the
 * summed device time; hf_profile_entry reads kind i (0 <= i < the count
 * returned); hf_profile_reset clears the totals.  Kinds: "splat", "passA",
 * "passB", "passB_fwd", "passC", "torque", "query", "resample", "y_tc"
 * (the tensor-core y stages of the precision variant), "passA_stationary"
 * (the x/y transforms of a stationary part's spectrum; "passB_fwd" is its z
 * transform). */
hf_status hf_profile_enable(hf_ctx *ctx, int on);
int hf_profile_read(hf_ctx *ctx);
hf_status hf_profile_entry(const hf_ctx *ctx, int i, const char **name, long long *launches,
                           double *total_ms);
void hf_profile_reset(hf_ctx *ctx);

/* ---- single-step entry points (each step of the path on its own) ---- */

/* Rotated resample (Section 2.4, motion decomposition):
 * d_out[n] = trilinear_periodic(d_rho, R^T x_n) for the 3x3 row-major h_R. */
hf_status hf_resample(int n, const float *d_rho, const float h_R[9], float *d_out, hf_stream stream);

/* Forward 3D real-to-complex DFT (Eq. 7a, unscaled, e^{-2 pi i k n / N}) of
 * d_in (N^3 floats, 8-byte aligned).  d_out: N x N x (N/2+1) complex64 as interleaved floats,
 * [kz][ky][kx] in natural frequency order.  d_scratch: at least
 * hf_rfft3d_scratch_bytes(n) bytes of device memory, 16-byte aligned. */
size_t hf_rfft3d_scratch_bytes(int n);
hf_status hf_rfft3d(int n, const float *d_in, float *d_out, void *d_scratch, hf_stream stream);

/* Energy and force for one rotation into explicit buffers (Eqs. 3, 5, 6a):
 * d_E, d_Fx, d_Fy, d_Fz are N^3 floats each (the force pointers may be NULL);
 * d_scratch: at least hf_fields_scratch_bytes(n) bytes, 16-byte aligned. */
size_t hf_fields_scratch_bytes(int n);
hf_status hf_fields(hf_ctx *ctx, const hf_part *s1, const hf_part *s2, const float h_quat[4],
                    float *d_E, float *d_Fx, float *d_Fy, float *d_Fz, void *d_scratch,
                    hf_stream stream);

/* Torque by least squares over the 6 nearest rotations for explicit
 * buffers: d_E is R x N^3, d_T is R x 3 x N^3, h_quat R x 4.  flags may hold
 * HF_TORQUE_F64 or HF_TORQUE_C.  h_status (R ints, may be NULL) receives 0 or 1 (rank
 * deficient: NaN torque).  Errors: HF_EINVAL (R < 7 or a rank-deficient
 * rotation), HF_ENOMEM, HF_ECUDA. */
hf_status hf_torque(hf_ctx *ctx, int n, int R, const float *h_quat, const float *d_E, float *d_T,
                    unsigned flags, int *h_status, hf_stream stream);

/* ---- energy and force without device allocation ----
 * The paper has no counterpart: this entry point exists for callers that may
 * not allocate device memory while they run -- a 1 kHz haptic loop, where a
 * cudaMalloc/cudaFree can stall the device well past the frame budget; a
 * plug-in whose host application owns all device memory; a runtime that
 * forbids allocation after start-up.  It computes what hf_fields computes
 * (energy and force of the rotated moving density against the stationary
 * one, for one rotation) directly from the two caller-owned N^3 grids d_rho1
 * (stationary) and d_rho2 (moving) into the caller-owned N^3 outputs (all
 * four required), and allocates nothing: its intermediates live in one
 * static device array of HF_NOALLOC_MAX_N-sized buffers (about 4.3 MB) that
 * every GPU loading the library holds until the process exits.
 *   - N must be 32 or 64 (N > HF_NOALLOC_MAX_N: HF_EINVAL with a message).
 *   - All calls share that array: calls whose GPU work overlaps (other
 *     streams or threads) race and give wrong results; order them.
 *   - The first call on a device is its set-up and is NOT allocation-free:
 *     CUDA loads device code lazily, so that call loads the library's
 *     kernels and the array onto the device (reserving the array), resolves
 *     the array's address and sets kernel attributes, with that device
 *     current.  Make one warm-up call per device at start-up, before the
 *     time-critical loop and before any stream capture; later calls
 *     allocate nothing.
 * Errors: HF_EINVAL, HF_ECUDA (message in hf_last_error()). */
#define HF_NOALLOC_MAX_N 64
hf_status hf_fields_noalloc(int n, const float *d_rho1, const float *d_rho2, const float h_quat[4],
                            float *d_E, float *d_Fx, float *d_Fy, float *d_Fz, hf_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* HF_H */
