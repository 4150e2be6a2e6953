// hf_kernels.cu -- the non-FFT steps of the path:
//   splat    skeletal density from skeleton samples (stand-in for the
//            skeletal density of Section 2.3, Gaussian kernel)
//   resample rotated density on the grid (Section 2.4)
//   torque   rotational gradient of the energy by least squares over the
//            nearest sampled rotations (the quantity of Eq. 6b)
//   query    fields at a pose from the per-orientation precompute
//            (Section 4.2, restricted motion DOF)
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "hf_internal.h"
#include "hf_sample.cuh"

namespace hf {

// ------------------------------------------------------------------ splat
// One CTA per 8x8x8 tile of nodes; each thread owns the two nodes lz and
// lz + 4 of its (lx, ly) column.  The CTA walks the point list in chunks,
// keeps (in point order) the points whose cutoff sphere reaches the tile's
// box, and every thread adds their Gaussians to its nodes.  Gather form:
// deterministic, no atomics.
//
// A kept point is stored as its offset from the tile centre, taken at its
// periodic image nearest that centre; a node's own offset from the centre,
// (l - 3.5) h per axis, is exact.  When the cutoff radius c and the tile's
// half-width w satisfy c + w < 1 (half the period), every node within c of
// the point sees it at that same image, and any other node lies beyond c at
// any image, so the node-point distance is one subtraction per axis.  A
// chunk holding a point with a cutoff too wide for that takes the minimum
// image per node instead.
//
// The two nodes' arithmetic runs as paired FP32 instructions (sm_100 add,
// multiply and fma on a float2, each half rounded as the scalar operation):
// the same operations in the same order per node as one node per thread,
// so the same bits.  The kept points are stored with their offsets negated
// and duplicated into pairs, so that no pair needs assembling.
constexpr int kSplatTile = 8;
constexpr int kSplatThreads = kSplatTile * kSplatTile * kSplatTile / 2;

__device__ __forceinline__ float min_image(float d) { return d - 2.0f * rintf(0.5f * d); }

// 2^t for t <= 0 down to -30 (the arguments here): the PTX base-2
// exponential, relative error within 2^-22 (its documented bound)
__device__ __forceinline__ float exp2_neg(float t) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(t));
    return r;
}

template <int N>
__global__ void __launch_bounds__(kSplatThreads, 6) splat_kernel(const float *__restrict__ pts,
                                                              const float *__restrict__ sigma,
                                                              const float *__restrict__ amp, int P,
                                                              float *__restrict__ grid) {
    // kept points: (-x, -x, -y, -y) and (-z, -z, a, a) of the offset from the
    // tile centre and the amplitude; (c^2, c^2, k, k) with c the cutoff and
    // k = -log2(e) / (2 sigma^2)
    __shared__ float4 cxy[kSplatThreads], cza[kSplatThreads], cpar[kSplatThreads];
    __shared__ int warp_cnt[kSplatThreads / 32];
    constexpr int TPA = N / kSplatTile;  // tiles per axis
    constexpr int HZ = kSplatTile / 2;   // the thread's second node is HZ further along z
    constexpr float kLog2e = 1.4426950408889634f;
    const int t = blockIdx.x;
    const int tx = t % TPA, ty = (t / TPA) % TPA, tz = t / (TPA * TPA);
    const float h = 2.0f / N;
    const int lx = threadIdx.x % kSplatTile, ly = (threadIdx.x / kSplatTile) % kSplatTile,
              lz = threadIdx.x / (kSplatTile * kSplatTile);
    const int nx = tx * kSplatTile + lx, ny = ty * kSplatTile + ly, nz = tz * kSplatTile + lz;
    // tile box: centre and half-width per axis; node offsets from the centre
    const float half = 0.5f * (kSplatTile - 1) * h;
    const float bx = (float)(tx * kSplatTile - N / 2) * h + half;
    const float by = (float)(ty * kSplatTile - N / 2) * h + half;
    const float bz = (float)(tz * kSplatTile - N / 2) * h + half;
    const float qx = (float)(2 * lx - (kSplatTile - 1)) * (0.5f * h);
    const float qy = (float)(2 * ly - (kSplatTile - 1)) * (0.5f * h);
    const float qz0 = (float)(2 * lz - (kSplatTile - 1)) * (0.5f * h);
    const float qz1 = (float)(2 * (lz + HZ) - (kSplatTile - 1)) * (0.5f * h);
    const float2 qx2 = make_float2(qx, qx), qy2 = make_float2(qy, qy), qz2 = make_float2(qz0, qz1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float2 acc = make_float2(0.0f, 0.0f);
    for (int base = 0; base < P; base += kSplatThreads) {
        const int i = base + threadIdx.x;
        bool keep = false, wide = false;
        float4 c = make_float4(0, 0, 0, 0);
        float2 cp = make_float2(0, 0);
        if (i < P) {
            const float s = __ldg(sigma + i);
            const float cut = 6.0f * s;
            c = make_float4(min_image(__ldg(pts + 3 * i) - bx), min_image(__ldg(pts + 3 * i + 1) - by),
                            min_image(__ldg(pts + 3 * i + 2) - bz), amp ? __ldg(amp + i) : 1.0f);
            // distance from the point to the tile box on the torus, per axis
            const float dx = fmaxf(fabsf(c.x) - half, 0.f);
            const float dy = fmaxf(fabsf(c.y) - half, 0.f);
            const float dz = fmaxf(fabsf(c.z) - half, 0.f);
            keep = dx * dx + dy * dy + dz * dz <= cut * cut * 1.0001f + 1e-12f;
            wide = keep && !(cut + half < 0.99f);
            cp = make_float2(36.0f * s * s, -kLog2e / (2.0f * s * s));
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) warp_cnt[warp] = __popc(m);
        const bool any_wide = __syncthreads_or(wide);
        int off = 0, total = 0;
        for (int wv = 0; wv < kSplatThreads / 32; ++wv) {
            const int cnt = warp_cnt[wv];
            off += (wv < warp) ? cnt : 0;
            total += cnt;
        }
        if (keep) {
            const int pos = off + __popc(m & ((1u << lane) - 1u));
            cxy[pos] = make_float4(-c.x, -c.x, -c.y, -c.y);
            cza[pos] = make_float4(-c.z, -c.z, c.w, c.w);
            cpar[pos] = make_float4(cp.x, cp.x, cp.y, cp.y);
        }
        __syncthreads();
        if (!any_wide) {
#pragma unroll 4
            for (int j = 0; j < total; ++j) {
                const float4 a = cxy[j], b = cza[j], pj = cpar[j];
                const float2 dx = __fadd2_rn(qx2, make_float2(a.x, a.y));
                const float2 dy = __fadd2_rn(qy2, make_float2(a.z, a.w));
                const float2 dz = __fadd2_rn(qz2, make_float2(b.x, b.y));
                const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
                const float2 e = __fmul2_rn(r2, make_float2(pj.z, pj.w));
                const float2 g = make_float2(exp2_neg(e.x), exp2_neg(e.y));
                const float2 w = make_float2(r2.x <= pj.x ? b.z : 0.0f, r2.y <= pj.y ? b.w : 0.0f);
                acc = __ffma2_rn(w, g, acc);
            }
        } else {
            for (int j = 0; j < total; ++j) {
                const float4 a = cxy[j], b = cza[j], pj = cpar[j];
                const float dx = min_image(qx + a.x), dy = min_image(qy + a.z);
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const float dz = min_image((k ? qz1 : qz0) + b.x);
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    if (r2 <= pj.x) {
                        const float v = fmaf(b.z, exp2_neg(r2 * pj.z), k ? acc.y : acc.x);
                        if (k) acc.y = v;
                        else acc.x = v;
                    }
                }
            }
        }
        __syncthreads();
    }
    grid[((size_t)nz * N + ny) * N + nx] = acc.x;
    grid[((size_t)(nz + HZ) * N + ny) * N + nx] = acc.y;
}

// --------------------------------------------------------------- resample
template <int N>
__global__ void resample_kernel(const float *__restrict__ rho, Rot9 rot, float *__restrict__ out) {
    const size_t total = (size_t)N * N * N;
    const float *R = rot.r;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % N), y = (int)((i / N) % N), z = (int)(i / ((size_t)N * N));
        const float cx = (float)(x - N / 2), cy = (float)(y - N / 2), cz = (float)(z - N / 2);
        const float vx = fmaf(R[0], cx, fmaf(R[3], cy, R[6] * cz));
        const float vy = fmaf(R[1], cx, fmaf(R[4], cy, R[7] * cz));
        const float vz = fmaf(R[2], cx, fmaf(R[5], cy, R[8] * cz));
        out[i] = trilinear_c<N>(rho, vx, vy, vz);
    }
}

// ----------------------------------------------------------------- torque
// T_i = -P_i (E_nb - E_i) per cell, P_i = (A^T A)^{-1} A^T (3 x 6, from the
// host in float64), A rows = Log(R_j R_i^T).  Blocks are ordered rotation-
// fastest over cell tiles so that one tile of every rotation's energy stays
// in L2 while all rotations that use it run.
constexpr int kTorqueThreads = 256;
constexpr int kTorqueVec = 2;  // float4 groups of cells per thread, all loads in flight together
constexpr int kTorqueTile = kTorqueThreads * 4 * kTorqueVec;

// The 3 x 6 least-squares product T_d = -sum_s P_ds (E_s - E_r) per cell, in
// one of three precisions (MODE): 0 float32 fma; 1 float64 over the float32
// differences; 2 compensated float32, as accurate as float64 before the final
// rounding.  Mode 2 is the dot product Dot2 of Ogita, Rump and Oishi
// ("Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005) with the
// float64 operator split into P = hi + lo (hi its float32 rounding, lo the
// float32 rounding of the rest, together within 2^-48 of P): each hi b is
// split exactly into its rounded product and the product's error (one fma),
// the rounded products are summed with TwoSum (Knuth) keeping every
// rounding error, and the errors, the lo b terms and the TwoSum errors are
// summed in float32 beside; the result is the float32 rounding of the two
// sums' total.  Its float32 arithmetic runs as paired instructions over the
// (x, y) and (z, w) cells of each float4 group.
template <int MODE>
__global__ void __launch_bounds__(kTorqueThreads) torque_kernel(const float *__restrict__ E, size_t es,
                                                                float *__restrict__ T, size_t ts,
                                                                const int *__restrict__ nbr,
                                                                const float *__restrict__ P,
                                                                const double *__restrict__ P64, int R,
                                                                size_t n3) {
    const int r = blockIdx.x % R;
    const size_t tile = blockIdx.x / R;
    __shared__ float2 s_hi[18], s_lo[18];
    if constexpr (MODE == 2) {
        // the rotation's operator as hi + lo, once per block (18 float64 subtractions)
        if (threadIdx.x < 18) {
            const float hi = __ldg(P + 18 * r + threadIdx.x);
            const float lo = (float)(__ldg(P64 + 18 * r + threadIdx.x) - (double)hi);
            s_hi[threadIdx.x] = make_float2(hi, hi);
            s_lo[threadIdx.x] = make_float2(lo, lo);
        }
        __syncthreads();
    }
    // group j of the thread covers cells c0 + 4 (j kTorqueThreads) .. + 3: a
    // warp's accesses stay contiguous for every j
    const size_t c0 = tile * kTorqueTile + (size_t)threadIdx.x * 4;
    int nb[6];
#pragma unroll
    for (int s = 0; s < 6; ++s) nb[s] = __ldg(nbr + 6 * r + s);
    float4 ei[kTorqueVec], ej[kTorqueVec][6];
    bool live[kTorqueVec];
#pragma unroll
    for (int j = 0; j < kTorqueVec; ++j) {
        const size_t c = c0 + (size_t)j * kTorqueThreads * 4;
        live[j] = c < n3;  // n3 is a multiple of 4
        if (live[j]) {
            ei[j] = __ldg(reinterpret_cast<const float4 *>(E + (size_t)r * es + c));
#pragma unroll
            for (int s = 0; s < 6; ++s) ej[j][s] = __ldg(reinterpret_cast<const float4 *>(E + (size_t)nb[s] * es + c));
        }
    }
#pragma unroll
    for (int j = 0; j < kTorqueVec; ++j) {
        if (!live[j]) continue;
        const size_t c = c0 + (size_t)j * kTorqueThreads * 4;
        float4 g[3];
        if constexpr (MODE == 2) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {  // the float4's (x, y) and (z, w) cells
                float2 b[6];
#pragma unroll
                for (int s = 0; s < 6; ++s) {
                    const float4 &u = ej[j][s];
                    const float2 a = h ? make_float2(u.z, u.w) : make_float2(u.x, u.y);
                    const float2 e0 = h ? make_float2(ei[j].z, ei[j].w) : make_float2(ei[j].x, ei[j].y);
                    b[s] = __fadd2_rn(a, make_float2(-e0.x, -e0.y));
                }
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    float2 p = make_float2(0.f, 0.f), c = make_float2(0.f, 0.f);
#pragma unroll
                    for (int s = 0; s < 6; ++s) {
                        const float2 hi = s_hi[6 * d + s], lo = s_lo[6 * d + s];
                        const float2 t = __fmul2_rn(hi, b[s]);                                // rounded hi b
                        const float2 e = __ffma2_rn(hi, b[s], make_float2(-t.x, -t.y));       // its exact error
                        if (s == 0) {
                            p = t;
                            c = __ffma2_rn(lo, b[s], e);
                        } else {
                            // TwoSum: p + t = ps + q exactly
                            const float2 ps = __fadd2_rn(p, t);
                            const float2 bv = __fadd2_rn(ps, make_float2(-p.x, -p.y));
                            const float2 av = __fadd2_rn(ps, make_float2(-bv.x, -bv.y));
                            const float2 q = __fadd2_rn(__fadd2_rn(p, make_float2(-av.x, -av.y)),
                                                        __fadd2_rn(t, make_float2(-bv.x, -bv.y)));
                            p = ps;
                            c = __fadd2_rn(c, __fadd2_rn(q, e));
                            c = __ffma2_rn(lo, b[s], c);
                        }
                    }
                    const float2 v = __fadd2_rn(p, c);
                    if (h) {
                        g[d].z = v.x;
                        g[d].w = v.y;
                    } else {
                        g[d].x = v.x;
                        g[d].y = v.y;
                    }
                }
            }
        } else if constexpr (MODE == 0) {
#pragma unroll
            for (int d = 0; d < 3; ++d) g[d] = make_float4(0, 0, 0, 0);
#pragma unroll
            for (int s = 0; s < 6; ++s) {
                const float4 b = make_float4(ej[j][s].x - ei[j].x, ej[j][s].y - ei[j].y, ej[j][s].z - ei[j].z,
                                             ej[j][s].w - ei[j].w);
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const float w = __ldg(P + 18 * r + 6 * d + s);
                    g[d].x = fmaf(w, b.x, g[d].x);
                    g[d].y = fmaf(w, b.y, g[d].y);
                    g[d].z = fmaf(w, b.z, g[d].z);
                    g[d].w = fmaf(w, b.w, g[d].w);
                }
            }
        } else {
            // the 3 x 6 product in float64 over float32 differences: a
            // difference of two float32 energies within a factor of two of
            // each other (neighbouring rotations, the common case) is exact in
            // float32 (Sterbenz), and otherwise carries one rounding of at
            // most 2^-24 of itself; the float64 pipe then does 18 fma per cell
            // instead of 6 subtractions more
            double gd[3][4] = {};
#pragma unroll
            for (int s = 0; s < 6; ++s) {
                const double b[4] = {(double)(ej[j][s].x - ei[j].x), (double)(ej[j][s].y - ei[j].y),
                                     (double)(ej[j][s].z - ei[j].z), (double)(ej[j][s].w - ei[j].w)};
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const double w = __ldg(P64 + 18 * r + 6 * d + s);
#pragma unroll
                    for (int q = 0; q < 4; ++q) gd[d][q] = fma(w, b[q], gd[d][q]);
                }
            }
#pragma unroll
            for (int d = 0; d < 3; ++d)
                g[d] = make_float4((float)gd[d][0], (float)gd[d][1], (float)gd[d][2], (float)gd[d][3]);
        }
#pragma unroll
        for (int d = 0; d < 3; ++d)
            *reinterpret_cast<float4 *>(T + (size_t)r * ts + (size_t)d * n3 + c) =
                make_float4(-g[d].x, -g[d].y, -g[d].z, -g[d].w);
    }
}

// ------------------------------------------------------------------ query
// One warp per query.  Rotation search in float64 (ordering by |q . q_j|,
// which orders the geodesic angle; ties to the lower index), weights
// 1/theta in float64, trilinear sampling in float32.
constexpr int kQueryMaxK = 8;
constexpr int kQueryWarps = 8;

__device__ __forceinline__ bool better(double da, int ia, double db, int ib) {
    return da > db || (da == db && ia < ib);
}

// Loads of the field sets by the queries: through L1 in a kernel launched
// after the set was built, at L2 (.cg) in the resident query kernel, which
// outlives builds that may reuse the addresses of sets it read earlier.
template <bool CG, class T>
__device__ __forceinline__ T ld_set(const T *p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// A double in [-1, 1] as a float by truncation, in integer operations (a
// float64-to-float32 conversion runs at the float64 rate): within 2^-23 of
// |x|; values below float's normal range read as zero.
__device__ __forceinline__ float f32_trunc(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned e = (hi >> 20) & 0x7ffu;
    if (e < 897u) return 0.0f;
    return __uint_as_float((hi & 0x80000000u) | ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}

// One query by one warp: `in` = (t, q), 7 results to `outp`.
template <int N, bool CG = false>
__device__ __forceinline__ void query_warp(const QueryGeom &g, const float *in, int k, float *outp,
                                           float *part) {
    const int lane = threadIdx.x & 31;
    double q[4] = {in[3], in[4], in[5], in[6]};
    const double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
#pragma unroll
    for (int a = 0; a < 4; ++a) q[a] /= qn;
    // The k nearest rotations by |<q, q_j>| (ties to the lower index), ranked
    // in float64.  A float64 warp instruction takes many times a float32
    // one, so in the launched kernels a float32 pass first finds the k-th
    // largest |dot| (K32), and
    // the float64 ranking then takes only rotations whose float32 |dot| is at
    // least K32 - 3e-6.  That keeps every rotation the float64 ranking can
    // select: the float32 |dot| is within 6 2^-24 of the float64 one (unit
    // quaternions, inputs truncated to float32 within 2^-23, four rounded
    // fmas), so the float64 k-th largest D >= K32 - 1e-6 and each selected
    // rotation's float32 |dot| >= D - 1e-6.  The selection, and so the result,
    // is the same as ranking every rotation in float64.
    const float qf[4] = {f32_trunc(q[0]), f32_trunc(q[1]), f32_trunc(q[2]), f32_trunc(q[3])};
    constexpr int kQueryLoads = 4;  // a lane's rotations j = lane + 32 i, loaded kQueryLoads at a time
    auto dot32 = [&](const double *v) {
        return fminf(fabsf(fmaf(qf[0], f32_trunc(v[0]),
                                fmaf(qf[1], f32_trunc(v[1]), fmaf(qf[2], f32_trunc(v[2]), qf[3] * f32_trunc(v[3]))))),
                     1.0f);
    };
    float tk[kQueryMaxK];  // this lane's k largest float32 |dot|, descending
#pragma unroll
    for (int s = 0; s < kQueryMaxK; ++s) tk[s] = -1.0f;
    double bd[kQueryMaxK];
    int bi[kQueryMaxK];
#pragma unroll
    for (int s = 0; s < kQueryMaxK; ++s) { bd[s] = -1.0; bi[s] = 0x7fffffff; }
    auto rank64 = [&](const double *v, int j) {  // insert into the lane's float64 top-k
        double d = fabs(q[0] * v[0] + q[1] * v[1] + q[2] * v[2] + q[3] * v[3]);
        d = fmin(d, 1.0);
        int ij = j;
#pragma unroll
        for (int s = 0; s < kQueryMaxK; ++s) {
            if (s < k && better(d, ij, bd[s], bi[s])) {
                const double td = bd[s];
                const int ti = bi[s];
                bd[s] = d; bi[s] = ij; d = td; ij = ti;
            }
        }
    };
    if constexpr (CG) {
        // the resident query kernel ranks every rotation in float64, one at a
        // time: its loads go to L2 (a second pass would pay them again), and
        // on an SM shared with the builds' float32 kernels the float64 pipe is
        // the idle one (measured: p50 47 us in serving against 62-68 us with
        // either float32-first form)
        for (int j = lane; j < g.R; j += 32) {
            const double *qj = g.quats + 4 * (size_t)j;
            const double v[4] = {ld_set<CG>(qj), ld_set<CG>(qj + 1), ld_set<CG>(qj + 2), ld_set<CG>(qj + 3)};
            rank64(v, j);
        }
    } else {
        for (int j0 = lane; j0 < g.R; j0 += 32 * kQueryLoads) {
            double qv[kQueryLoads][4];
#pragma unroll
            for (int u = 0; u < kQueryLoads; ++u) {
                const int j = j0 + 32 * u;
                if (j < g.R) {
                    const double *qj = g.quats + 4 * (size_t)j;
#pragma unroll
                    for (int a = 0; a < 4; ++a) qv[u][a] = ld_set<CG>(qj + a);
                }
            }
#pragma unroll
            for (int u = 0; u < kQueryLoads; ++u) {
                if (j0 + 32 * u >= g.R) break;
                float df = dot32(qv[u]);
#pragma unroll
                for (int s = 0; s < kQueryMaxK; ++s)
                    if (s < k && df > tk[s]) {
                        const float t = tk[s];
                        tk[s] = df;
                        df = t;
                    }
            }
        }
        float kth = -1.0f;  // the warp's k-th largest float32 |dot|
        for (int s = 0; s < k; ++s) {
            float v = tk[0];
            int owner = lane;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float ov = __shfl_xor_sync(0xffffffffu, v, o);
                const int oo = __shfl_xor_sync(0xffffffffu, owner, o);
                if (ov > v || (ov == v && oo < owner)) { v = ov; owner = oo; }
            }
            kth = v;
            if (owner == lane) {
#pragma unroll
                for (int t = 0; t < kQueryMaxK - 1; ++t) tk[t] = tk[t + 1];
                tk[kQueryMaxK - 1] = -1.0f;
            }
        }
        const float tau = kth - 3e-6f;
        // per-lane sorted top-k of (|dot|, index) over the candidates, in float64;
        // lanes visit indices in ascending order
        for (int j0 = lane; j0 < g.R; j0 += 32 * kQueryLoads) {
            double qv[kQueryLoads][4];
#pragma unroll
            for (int u = 0; u < kQueryLoads; ++u) {
                const int j = j0 + 32 * u;
                if (j < g.R) {
                    const double *qj = g.quats + 4 * (size_t)j;
#pragma unroll
                    for (int a = 0; a < 4; ++a) qv[u][a] = ld_set<CG>(qj + a);
                }
            }
#pragma unroll
            for (int u = 0; u < kQueryLoads; ++u) {
                const int j = j0 + 32 * u;
                if (j >= g.R) break;
                if (dot32(qv[u]) >= tau) rank64(qv[u], j);
            }
        }
    }  // two passes
    // warp merge: k rounds of arg-best over the lanes' list heads
    double sel_d[kQueryMaxK];
    int sel_i[kQueryMaxK];
    for (int s = 0; s < k; ++s) {
        double d = bd[0];
        int i = bi[0];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double od = __shfl_xor_sync(0xffffffffu, d, o);
            const int oi = __shfl_xor_sync(0xffffffffu, i, o);
            if (better(od, oi, d, i)) { d = od; i = oi; }
        }
        sel_d[s] = d;
        sel_i[s] = i;
        if (bi[0] == i) {  // this lane owned the winner: pop its head
#pragma unroll
            for (int t = 0; t < kQueryMaxK - 1; ++t) { bd[t] = bd[t + 1]; bi[t] = bi[t + 1]; }
            bd[kQueryMaxK - 1] = -1.0;
            bi[kQueryMaxK - 1] = 0x7fffffff;
        }
    }
    // weights 1/theta, theta = 2 acos(|dot|): lane s < k computes the s-th
    // theta, the others none (a float64 warp instruction costs per active lane)
    double th = 1.0;
#pragma unroll
    for (int s = 0; s < kQueryMaxK; ++s)
        if (s == lane && s < k) th = 2.0 * acos(sel_d[s]);
    double w[kQueryMaxK];
    int used = k;
    if (__shfl_sync(0xffffffffu, th < 1e-12 ? 1 : 0, 0)) {
        used = 1;
        w[0] = 1.0;
    } else {
        const double wl = lane < k ? 1.0 / th : 0.0;
        double sw = 0.0;
        for (int s = 0; s < k; ++s) { w[s] = __shfl_sync(0xffffffffu, wl, s); sw += w[s]; }
        for (int s = 0; s < k; ++s) w[s] /= sw;
    }
    // trilinear per (field, rotation) pair at lag u = t / h
    const float hinv = 0.5f * N;
    const float ux = in[0] * hinv, uy = in[1] * hinv, uz = in[2] * hinv;
    const float fx = floorf(ux), fy = floorf(uy), fz = floorf(uz);
    const float ax = ux - fx, ay = uy - fy, az = uz - fz;
    const int x0 = wrapN<N>((int)fx), y0 = wrapN<N>((int)fy), z0 = wrapN<N>((int)fz);
    const int x1 = wrapN<N>(x0 + 1), y1 = wrapN<N>(y0 + 1), z1 = wrapN<N>(z0 + 1);
    const size_t n3 = (size_t)N * N * N;
    for (int pidx = lane; pidx < 7 * used; pidx += 32) {
        const int f = pidx % 7, s = pidx / 7;
        float v = 0.f;
        if (g.field_slot[f] >= 0) {
            const float *fb = g.base + (size_t)sel_i[s] * g.rot_stride + (size_t)g.field_slot[f] * n3;
            const float *r00 = fb + ((size_t)z0 * N + y0) * N, *r01 = fb + ((size_t)z0 * N + y1) * N;
            const float *r10 = fb + ((size_t)z1 * N + y0) * N, *r11 = fb + ((size_t)z1 * N + y1) * N;
            const float v00 = ld_set<CG>(r00 + x0), v01 = ld_set<CG>(r01 + x0);
            const float v10 = ld_set<CG>(r10 + x0), v11 = ld_set<CG>(r11 + x0);
            const float c00 = fmaf(ax, ld_set<CG>(r00 + x1) - v00, v00);
            const float c01 = fmaf(ax, ld_set<CG>(r01 + x1) - v01, v01);
            const float c10 = fmaf(ax, ld_set<CG>(r10 + x1) - v10, v10);
            const float c11 = fmaf(ax, ld_set<CG>(r11 + x1) - v11, v11);
            const float c0 = fmaf(ay, c01 - c00, c00), c1 = fmaf(ay, c11 - c10, c10);
            v = fmaf(az, c1 - c0, c0);
        }
        part[pidx] = v * (float)w[s];
    }
    __syncwarp();
    if (lane < 7) {
        float acc = 0.f;
        for (int s = 0; s < used; ++s) acc += part[7 * s + lane];
        outp[lane] = acc;
    }
}

template <int N>
__global__ void query_kernel(QueryGeom g, const float *__restrict__ tq, int Q, int k, float *__restrict__ out) {
    __shared__ float part[kQueryWarps][7 * kQueryMaxK];
    const int warp = threadIdx.x >> 5;
    const int qi = blockIdx.x * kQueryWarps + warp;
    if (qi >= Q) return;  // warp-uniform
    query_warp<N>(g, tq + 7 * (size_t)qi, k, out + 7 * (size_t)qi, part[warp]);
}

// a single query whose pose travels as a kernel argument; `out` may be mapped
// host memory, so the answer needs no copy back
template <int N>
__global__ void query_one_kernel(QueryGeom g, Pose7 pose, int k, float *out) {
    __shared__ float part[7 * kQueryMaxK];
    query_warp<N>(g, pose.v, k, out, part);
}

// The resident query kernel: a query answered without a launch.  The host
// writes a lane's request (set geometry, pose, k) into the lane's mailbox in
// mapped pinned memory, then bumps the lane's request number in the mailbox
// header; warp 0 of the block polls the header, and the warp that serves the
// lane runs the query and writes the 7 results and the request's number back.
// An instance serves for `life_ns` of the global timer (or until *stop) and
// returns: every wait checks that deadline, so no instance outlives it by
// more than one query.  The host keeps the next instance queued on the same
// stream behind the running one.  served[] (device memory) carries each
// lane's last answered request number from one instance to the next.
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned ld_acquire_sys(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys(unsigned *p, unsigned v) {
    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <int N>
__device__ __noinline__ void query_resident_serve(const QueryReq &r, float *part, float *out) {
    query_warp<N, true>(r.g, r.pose.v, r.k, out, part);
}

__global__ void __launch_bounds__(32 * (kResidentLanesPerBlock + 1), 1)
    query_resident_kernel(QueryMail *mail, unsigned *req, unsigned *served, const unsigned *stop, int lanes,
                          unsigned long long life_ns, unsigned long long max_polls) {
    __shared__ volatile unsigned s_pend[kResidentLanesPerBlock];
    __shared__ volatile int s_quit;
    __shared__ float part[kResidentLanesPerBlock][7 * kQueryMaxK];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int base = blockIdx.x * kResidentLanesPerBlock;
    const int nl = min(kResidentLanesPerBlock, lanes - base);
    if (threadIdx.x < kResidentLanesPerBlock) s_pend[threadIdx.x] = 0u;
    if (threadIdx.x == 0) s_quit = 0;
    __syncthreads();
    const unsigned long long t_end = global_ns() + life_ns;
    if (warp == 0) {
        // the poller: lane j watches mailbox base + j
        unsigned last = lane < nl ? served[base + lane] : 0u;
        for (unsigned long long it = 0; it < max_polls; ++it) {
            // warp-uniform: every lane leaves the loop together
            if (__any_sync(0xffffffffu, global_ns() > t_end || ld_acquire_sys(stop) != 0u)) break;
            if (lane < nl && s_pend[lane] == 0u) {
                const unsigned cur = ld_acquire_sys(req + base + lane);
                if (cur != last) {
                    last = cur;
                    s_pend[lane] = cur;
                    __threadfence_block();
                }
            }
            __syncwarp();
            __nanosleep(256);
        }
        if (lane == 0) s_quit = 1;
        return;
    }
    const int j = warp - 1;  // the lane this warp serves
    if (j >= nl) return;
    QueryMail &m = mail[base + j];
    constexpr int kReqWords = sizeof(QueryReq) / 4;
    static_assert(sizeof(QueryReq) % 4 == 0 && kReqWords <= 32, "one request word per lane");
    // bounded by the poller's exit (s_quit); the iteration bound is a second
    // stop, looser than the poller's since a sleep may end early
    for (unsigned long long it = 0; it < 8 * max_polls; ++it) {
        const unsigned p = __shfl_sync(0xffffffffu, s_pend[j], 0);  // warp-uniform
        if (p != 0u) {
            __threadfence_block();  // the poller acquired the request's number before publishing it here
            // the request, one word per lane read past the caches, then gathered
            const unsigned wv = lane < kReqWords ? __ldcv(reinterpret_cast<const unsigned *>(&m.rq) + lane) : 0u;
            QueryReq r;
            unsigned *rw = reinterpret_cast<unsigned *>(&r);
#pragma unroll
            for (int w = 0; w < kReqWords; ++w) rw[w] = __shfl_sync(0xffffffffu, wv, w);
            float *out = m.out;
            switch (r.n) {
                case 32: query_resident_serve<32>(r, part[j], out); break;
                case 64: query_resident_serve<64>(r, part[j], out); break;
                case 96: query_resident_serve<96>(r, part[j], out); break;
                case 128: query_resident_serve<128>(r, part[j], out); break;
                case 256: query_resident_serve<256>(r, part[j], out); break;
                default:
                    if (lane < 7) out[lane] = __int_as_float(0x7fc00000);  // NaN: an unsupported size
            }
            __threadfence_system();  // each lane's results before the number that publishes them
            __syncwarp();
            if (lane == 0) {
                st_release_sys(&m.done, p);
                served[base + j] = p;
                s_pend[j] = 0u;
            }
            __syncwarp();
            continue;
        }
        if (__shfl_sync(0xffffffffu, s_quit, 0)) break;
        __nanosleep(128);
    }
}

cudaError_t launch_query_resident(QueryMail *mail, unsigned *req, unsigned *served, const unsigned *stop, int lanes,
                                  unsigned long long life_ns, cudaStream_t st) {
    if (lanes <= 0) return cudaErrorInvalidValue;
    const int blocks = (lanes + kResidentLanesPerBlock - 1) / kResidentLanesPerBlock;
    // an iteration bound besides the timer: at least 128 ns per poll
    const unsigned long long max_polls = life_ns / 128 + 1024;
    query_resident_kernel<<<blocks, 32 * (kResidentLanesPerBlock + 1), 0, st>>>(mail, req, served, stop, lanes,
                                                                              life_ns, max_polls);
    return cudaGetLastError();
}

// ------------------------------------------------------------- launchers
#define HF_DISPATCH_K(n, call)                              \
    switch (n) {                                            \
        case 32: { constexpr int NN = 32; call; break; }    \
        case 64: { constexpr int NN = 64; call; break; }    \
        case 96: { constexpr int NN = 96; call; break; }    \
        case 128: { constexpr int NN = 128; call; break; }  \
        case 256: { constexpr int NN = 256; call; break; }  \
        default: return cudaErrorInvalidValue;              \
    }

cudaError_t run_splat(int n, const float *pts, const float *sigma, const float *amp, int P, float *grid,
                      cudaStream_t st) {
    const int tiles = (n / kSplatTile) * (n / kSplatTile) * (n / kSplatTile);
    HF_DISPATCH_K(n, (splat_kernel<NN><<<tiles, kSplatThreads, 0, st>>>(pts, sigma, amp, P, grid)));
    return cudaGetLastError();
}

cudaError_t run_resample(int n, const float *rho, Rot9 rot, float *out, cudaStream_t st) {
    HF_DISPATCH_K(n, (resample_kernel<NN><<<4 * 148, 256, 0, st>>>(rho, rot, out)));
    return cudaGetLastError();
}

cudaError_t run_torque(int n, int R, const float *E, size_t e_rot_stride, float *T, size_t t_rot_stride,
                       const int *nbr, const float *P, const double *P64, int mode, cudaStream_t st) {
    const size_t n3 = (size_t)n * n * n;
    const size_t tiles = (n3 + kTorqueTile - 1) / kTorqueTile;
    const size_t blocks = tiles * (size_t)R;
    if (blocks > 0x7fffffffull) return cudaErrorInvalidValue;
    if (mode == 1)
        torque_kernel<1><<<(unsigned)blocks, kTorqueThreads, 0, st>>>(E, e_rot_stride, T, t_rot_stride, nbr, P, P64, R, n3);
    else if (mode == 2)
        torque_kernel<2><<<(unsigned)blocks, kTorqueThreads, 0, st>>>(E, e_rot_stride, T, t_rot_stride, nbr, P, P64, R, n3);
    else
        torque_kernel<0><<<(unsigned)blocks, kTorqueThreads, 0, st>>>(E, e_rot_stride, T, t_rot_stride, nbr, P, P64, R, n3);
    return cudaGetLastError();
}

cudaError_t run_query_one(const QueryGeom &g, Pose7 pose, int k, float *out, cudaStream_t st) {
    HF_DISPATCH_K(g.n, (query_one_kernel<NN><<<1, 32, 0, st>>>(g, pose, k, out)));
    return cudaGetLastError();
}

cudaError_t run_query(const QueryGeom &g, const float *tq, int Q, int k, float *out, cudaStream_t st) {
    if (Q <= 0) return cudaSuccess;
    const int blocks = (Q + kQueryWarps - 1) / kQueryWarps;
    HF_DISPATCH_K(g.n, (query_kernel<NN><<<blocks, 32 * kQueryWarps, 0, st>>>(g, tq, Q, k, out)));
    return cudaGetLastError();
}

// Never launched: its address names this file's device-code module, which
// hf_ctx_preload loads whole.
__global__ void module_anchor_kernels_kernel() {}
const void *module_anchor_kernels() { return (const void *)&module_anchor_kernels_kernel; }

}  // namespace hf
