// hf_fft.cu -- the per-rotation energy/force pipeline as three slab/pencil
// passes over an N^3 grid (Section 3.2: interpolate, multiply, inverse FFT;
// with the forward transform of the rotated density added because the
// resample is done in the spatial domain).
//
//   pass A  (one CTA per z-plane and rotation)
//           rho2^R = trilinear(rho2, R^T x_n)             Section 2.4
//           x: real-to-complex DFT of every row            Eq. 7a
//           y: complex DFT of every kx column              Eq. 7a
//           -> X1[r][z][ky*][kx*]     (* = digit-permuted slot order)
//   pass B  (one CTA per ky slot, kx chunk and rotation)
//           z: complex DFT of every (ky, kx) pencil        Eq. 7a
//           S  = (h^3/N^3) rho1^ . conj(rho2^R^)            Eqs. 3, 5
//           Gz = i pi kz~ S                                 Eq. 6a (2 pi w = pi k~)
//           z: inverse DFT of S and of Gz                   Eq. 7b
//           -> Y1 = S', Y2 = Gz'      [r][z][ky*][kx*]
//   pass C  (one CTA per z-plane and rotation)
//           Gy = i pi ky~ S'; y: inverse DFT of S', Gy, Gz' Eq. 7b
//           x: one complex inverse DFT per row gives two real fields:
//              IDFT(S (1 + pi kx~))  = E + i Fx   (Gx = i pi kx~ S)
//              IDFT(-(Gy + i Gz))    = Fy + i Fz
//           -> E, Fx, Fy, Fz (float, [z][y][x])
//
// The multipliers of Gx and Gy are constant along the pencils transformed
// before they are applied, so Gx needs no transform of its own until the
// last (x) stage and Gy none before pass C: 2 z-, 3 y- and 2 full x-
// transforms per rotation instead of the 4 of each that a field-by-field
// inverse takes.  Nyquist multipliers are 0 on every axis.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#include "hf_dft.cuh"
#include "hf_spec.cuh"
#include "hf_internal.h"
#include "hf_sample.cuh"

namespace hf {

template <int L>
__device__ __forceinline__ void load_tw(float2 *dst) {
    for (int i = threadIdx.x; i < L; i += blockDim.x) dst[i] = make_float2(g_tw<L>.v[i].x, g_tw<L>.v[i].y);
}

constexpr float kPi = 3.14159265358979323846f;

template <int N>
__device__ __forceinline__ float signed_k_mult(int k) {
    // pi * k~ with k~ the signed index, 0 at the Nyquist index
    return (2 * k == N) ? 0.0f : kPi * (float)(k < N / 2 ? k : k - N);
}

// ------------------------------------------------------------------ pass A
// Source of the plane: SRC_RAW samples a plain [z][y][x] grid at the rotated
// node positions (8 loads per trilinear sample); SRC_PLANES reads plane z of
// rotation r of an already resampled chunk rho2^R[r][z][y][x] (the identity
// rotation is this mode with r = 0) by asynchronous 8-byte copies.
// SRC_TEX samples through the texture units' 2x2 gathers (tex_resample).
enum { SRC_RAW = 0, SRC_PLANES = 1, SRC_TEX = 2 };

template <int N>
struct PassA {
    static constexpr int H = N / 2 + 1, HALF = N / 2;
    static constexpr int NT = (N >= 64) ? 256 : 128;
    static constexpr int MINB = (N >= 128) ? 3 : 4;
    static constexpr size_t smem = sizeof(float2) * ((size_t)N * H + N + HALF);
};

__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Bulk copies (the TMA engine's untiled form) into this CTA's shared memory,
// completing on an mbarrier; both addresses 16-byte aligned, bytes a
// multiple of 16.  Waits are bounded: a wait that gives up counts itself in
// g_bulk_timeouts (the blocks that read such a plane wrote invalid output).
__device__ int g_bulk_timeouts = 0;
constexpr unsigned long long kBulkWaitNs = 200ull * 1000 * 1000;

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init1(unsigned long long *mbar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\nfence.mbarrier_init.release.cluster;\n" ::"r"(smem_addr(mbar))
                 : "memory");
}
// the arrival that opens a phase expecting `bytes` of copies
__device__ __forceinline__ void mbar_expect(unsigned long long *mbar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)), "r"(bytes) : "memory");
}
// generic-proxy accesses to shared memory before this point are ordered before
// the async-proxy writes of copies issued after it (by this thread, after a
// barrier that covers the other threads' accesses)
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(mbar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long *mbar, unsigned parity) {
    unsigned ok;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(smem_addr(mbar)), "r"(parity)
                 : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// wait for phase `parity` of mbar; on giving up, count it and wait once more
// (bounded) so that no copy is left writing into the block's shared memory
__device__ __forceinline__ void mbar_wait_bounded(unsigned long long *mbar, unsigned parity) {
    for (int attempt = 0; attempt < 2; ++attempt) {
        const unsigned long long t0 = globaltimer_ns();
        while (!mbar_test(mbar, parity))
            if (globaltimer_ns() - t0 > kBulkWaitNs) break;
        if (mbar_test(mbar, parity)) return;
        if (attempt == 0 && threadIdx.x == 0) atomicAdd(&g_bulk_timeouts, 1);
    }
}

// The rotated resample through the texture units.  The moving grid is held as a
// 2D float array of stacked z-slices, each (N+1) x (N+1) with the wrapped
// row y = N and column x = N appended, so slice z spans rows
// [z(N+1), z(N+1)+N].  One 2x2 gather at the corner (x0 + 1, row0 + 1)
// returns texels (x0, x0+1) x (row0, row0+1) exactly (the footprint of an
// integer corner does not depend on the unit's coordinate rounding), so a
// trilinear sample is two gathers; the weights stay in float32 software.
template <int N>
struct TexSample {
    float4 a, b;       // gathers at slices z0 and z0 + 1
    float ax, ay, az;  // fractional offsets
};

// The support of the moving density as cell intervals, per axis a: a cell
// with lower corner c (corners c and c + 1, mod N) holds a nonzero node only
// if ((c - lo[a]) mod N) < len[a] (support_box_kernel).  Any other cell's
// eight corners are zero, and so is every sample in it.
struct CellBox {
    int lo[3], len[3];
};
template <int N>
__device__ __forceinline__ CellBox load_cell_box(const int *__restrict__ box) {
    CellBox b;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        b.lo[a] = box ? __ldg(box + 2 * a) : 0;
        b.len[a] = box ? __ldg(box + 2 * a + 1) : N;
    }
    return b;
}
template <int N>
__device__ __forceinline__ bool cell_in(int c, int lo, int len) {
    if constexpr ((N & (N - 1)) == 0) {
        return ((c - lo) & (N - 1)) < len;
    } else {
        int d = c - lo;
        d += d < 0 ? N : 0;
        return d < len;
    }
}

// Issue the two gathers of one sample; tex_combine waits for them.  Splitting
// the two lets a thread keep the gathers of several samples in flight.  A
// sample in a cell outside the support box issues none: its corners are all
// zero, and the zeros it combines give the +0 the gathers would.
template <int N>
__device__ __forceinline__ TexSample<N> tex_issue(cudaTextureObject_t t, float vx, float vy, float vz,
                                                  const CellBox &box) {
    constexpr int SC = TexLayout<N>::SC;
    TexSample<N> s;
    const float fx = floorf(vx), fy = floorf(vy), fz = floorf(vz);
    s.ax = vx - fx;
    s.ay = vy - fy;
    s.az = vz - fz;
    const int x0 = wrapN<N>((int)fx + N / 2), y0 = wrapN<N>((int)fy + N / 2), z0 = wrapN<N>((int)fz + N / 2);
    const int z1 = wrapN<N>(z0 + 1);
    const bool need = cell_in<N>(x0, box.lo[0], box.len[0]) & cell_in<N>(y0, box.lo[1], box.len[1]) &
                      cell_in<N>(z0, box.lo[2], box.len[2]);
    if (need) {
        // slice z sits at texel origin ((z % SC)(N+1), (z / SC)(N+1))
        // gather components: w = (x0, y0), z = (x0+1, y0), x = (x0, y0+1), y = (x0+1, y0+1)
        s.a = tex2Dgather<float4>(t, (float)((z0 % SC) * (N + 1) + x0) + 1.0f,
                                  (float)((z0 / SC) * (N + 1) + y0) + 1.0f, 0);
        s.b = tex2Dgather<float4>(t, (float)((z1 % SC) * (N + 1) + x0) + 1.0f,
                                  (float)((z1 / SC) * (N + 1) + y0) + 1.0f, 0);
    } else {
        s.a = s.b = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    return s;
}

template <int N>
__device__ __forceinline__ float tex_combine(const TexSample<N> &s) {
    const float4 a = s.a, b = s.b;
    const float a0 = fmaf(s.ax, a.z - a.w, a.w), a1 = fmaf(s.ax, a.y - a.x, a.x);
    const float b0 = fmaf(s.ax, b.z - b.w, b.w), b1 = fmaf(s.ax, b.y - b.x, b.x);
    const float c0 = fmaf(s.ay, a1 - a0, a0), c1 = fmaf(s.ay, b1 - b0, b0);
    return fmaf(s.az, c1 - c0, c0);
}

// Resample ROWS rows of the rotated grid, nodes (x, y0 + row, z) for x in
// [0, N), into reals at Pf[row * 2H + x] through the texture, U samples per
// thread in flight.  Sample i is node (i % N, i / N).  With COUNTERS (NT a
// multiple of N) a thread keeps one x and steps its row by NT / N: its node
// coordinates are float counters (exact small integers) instead of per-sample
// index arithmetic, and the x and z terms of R^T c are formed once, so a
// sample's position is one fma per axis (the same point, rounded in another
// order).
// The counters take more registers: pass A has them to spare, the pencil x
// forward (four CTAs per SM at 64 registers) does not.
constexpr int kTexInFlight = 8;
template <int N>
__device__ __forceinline__ float3 rotated_node(const float *R, float cx, float cy, float cz) {
    // (R^T c)_a = R[0][a] cx + R[1][a] cy + R[2][a] cz
    const float ax = fmaf(R[0], cx, R[3] * cy), ay = fmaf(R[1], cx, R[4] * cy), az = fmaf(R[2], cx, R[5] * cy);
    return make_float3(fmaf(R[6], cz, ax), fmaf(R[7], cz, ay), fmaf(R[8], cz, az));
}
template <int N, int NT, int ROWS, bool COUNTERS, int U = kTexInFlight>
__device__ __forceinline__ void tex_resample(cudaTextureObject_t t, const float *R, float *Pf, const int *box, int y0,
                                             int z) {
    constexpr int H = N / 2 + 1, COUNT = ROWS * N;
    const CellBox cb = load_cell_box<N>(box);
    const float cz = (float)(z - N / 2);
    if constexpr (COUNTERS && NT % N == 0) {
        constexpr int RS = NT / N;  // rows per step of a thread
        const int x = threadIdx.x % N, row0 = threadIdx.x / N;
        const float cx = (float)(x - N / 2);
        float cy = (float)(y0 + row0 - N / 2);
        float *dst = Pf + row0 * 2 * H + x;
        // the thread's fixed x and z terms of R^T c, so that a sample adds R[1][a] cy in one fma
        const float bx = fmaf(R[6], cz, R[0] * cx), by = fmaf(R[7], cz, R[1] * cx), bz = fmaf(R[8], cz, R[2] * cx);
#pragma unroll 1
        for (int i0 = threadIdx.x; i0 < COUNT; i0 += NT * U) {
            TexSample<N> s[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (COUNT % (NT * U) == 0 || i0 + u * NT < COUNT) {
                    const float cyu = cy + (float)(u * RS);
                    s[u] = tex_issue<N>(t, fmaf(R[3], cyu, bx), fmaf(R[4], cyu, by), fmaf(R[5], cyu, bz), cb);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (COUNT % (NT * U) == 0 || i0 + u * NT < COUNT) dst[u * RS * 2 * H] = tex_combine<N>(s[u]);
            cy += (float)(U * RS);
            dst += U * RS * 2 * H;
        }
    } else {
#pragma unroll 1
        for (int i0 = threadIdx.x; i0 < COUNT; i0 += NT * U) {
            TexSample<N> s[U];
            int dst[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = i0 + u * NT;
                if (COUNT % (NT * U) == 0 || i < COUNT) {
                    const int x = i % N, row = i / N;
                    const float3 v = rotated_node<N>(R, (float)(x - N / 2), (float)(y0 + row - N / 2), cz);
                    s[u] = tex_issue<N>(t, v.x, v.y, v.z, cb);
                    dst[u] = row * 2 * H + x;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (COUNT % (NT * U) == 0 || i0 + u * NT < COUNT) Pf[dst[u]] = tex_combine<N>(s[u]);
        }
    }
}

// The body of one pass A block, plane z of rotation r (a kernel's blockIdx
// or a persistent kernel's work item); sm is the block's dynamic shared memory.
template <int N, int SRC>
__device__ __forceinline__ void passA_body(const float *__restrict__ rho, const float *__restrict__ rot9,
                                           float2 *__restrict__ X1, cudaTextureObject_t tex,
                                           const int *__restrict__ box, unsigned zu, unsigned ru) {
    __builtin_assume(zu < (1u << 16) && ru < (1u << 16));  // the ranges of the blockIdx they stand for
    const int z = (int)zu, r = (int)ru;
    constexpr int H = PassA<N>::H, HALF = PassA<N>::HALF, NT = PassA<N>::NT;
    extern __shared__ __align__(16) float2 sm[];
    float2 *P = sm;            // [N rows y][H]  (row = N reals = N/2 complex + Nyquist slot)
    float2 *twN = P + N * H;   // exp(-2 pi i j / N)
    float2 *twH = twN + N;     // exp(-2 pi i j / (N/2))
    float *Pf = reinterpret_cast<float *>(P);

    if constexpr (SRC == SRC_PLANES) {
        const float2 *src = reinterpret_cast<const float2 *>(rho + ((size_t)r * N + z) * N * N);
        for (int i = threadIdx.x; i < N * N / 2; i += NT) {
            const int y = i / (N / 2), x2 = i % (N / 2);
            cp_async8(P + (size_t)y * H + x2, src + i);
        }
        load_tw<N>(twN);
        load_tw<HALF>(twH);
        cp_async_wait_all();
    } else {
        load_tw<N>(twN);
        load_tw<HALF>(twH);
        // rotated resample of the moving density into the plane, as reals
        float R[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) R[k] = __ldg(rot9 + 9 * r + k);
        if constexpr (SRC == SRC_TEX) {
            tex_resample<N, NT, N, true>(tex, R, Pf, box, 0, z);
        } else {
            const float cz = (float)(z - N / 2);
            const float bx = R[6] * cz, by = R[7] * cz, bz = R[8] * cz;
            for (int i = threadIdx.x; i < N * N; i += NT) {
                const int x = i % N, y = i / N;
                const float cx = (float)(x - N / 2), cy = (float)(y - N / 2);
                // (R^T c)_a = R[0][a] cx + R[1][a] cy + R[2][a] cz
                const float vx = fmaf(R[0], cx, fmaf(R[3], cy, bx));
                const float vy = fmaf(R[1], cx, fmaf(R[4], cy, by));
                const float vz = fmaf(R[2], cx, fmaf(R[5], cy, bz));
                Pf[(size_t)y * 2 * H + x] = trilinear_c<N>(rho, vx, vy, vz);
            }
        }
    }
    __syncthreads();

    // x: rows as N/2-point complex sequences z[m] = x[2m] + i x[2m+1]
    fft_lines<HALF, -1, N, 1, H, NT>(P, twH);
    // split into the half spectrum X[k], k = 0..N/2:
    //   E_k = (Z[k] + conj Z[N/2-k]) / 2,  O_k = (Z[k] - conj Z[N/2-k]) / 2i
    //   X[k] = E_k + W^k O_k,  X[N/2-k] = conj(E_k - W^k O_k),  W = exp(-2 pi i / N)
    for (int i = threadIdx.x; i < N * (N / 4 + 1); i += NT) {
        const int y = i % N, k = i / N;
        float2 *row = P + y * H;
        if (k == 0) {
            // X[0] and X[N/2] are real: packed as X[0] + i X[N/2] for the y transform
            const float2 z0 = row[0];
            row[0] = make_float2(z0.x + z0.y, z0.x - z0.y);
        } else if (4 * k == N) {
            const int s = perm_slot<HALF>(k);
            row[s] = cconj(row[s]);
        } else {
            const int s1 = perm_slot<HALF>(k), s2 = perm_slot<HALF>(HALF - k);
            const float2 a = row[s1], b = row[s2];
            const float2 Ek = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
            const float2 Ok = make_float2(0.5f * (a.y + b.y), -0.5f * (a.x - b.x));
            const float2 WO = cmul(tw_pick<N, N % 32 == 0>(twN, k), Ok);  // k = i / N: warp-uniform
            row[s1] = cadd(Ek, WO);
            row[s2] = cconj(csub(Ek, WO));
        }
    }
    __syncthreads();
    // y: the N/2 columns 0..N/2-1 of length N, column 0 carrying the real
    // columns kx = 0 and kx = N/2 as one complex sequence
    fft_lines<N, -1, HALF, H, 1, NT>(P, twN);
    // separate them: with Z = Y0 + i YN (Y0, YN transforms of real columns),
    // Y0[k] = (Z[k] + conj Z[-k]) / 2 and YN[k] = -i (Z[k] - conj Z[-k]) / 2;
    // thread k < N/2 + 1 owns the slots of k and N - k
    if (threadIdx.x <= HALF) {
        const int k = threadIdx.x;
        const int sa = perm_slot<N>(k), sb = perm_slot<N>((N - k) % N);
        const float2 a = P[sa * H], b = P[sb * H];
        const float2 y0 = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
        const float2 yn = make_float2(0.5f * (a.y + b.y), -0.5f * (a.x - b.x));
        P[sa * H] = y0;
        P[sa * H + HALF] = yn;
        if (sb != sa) {
            P[sb * H] = cconj(y0);
            P[sb * H + HALF] = cconj(yn);
        }
    }
    __syncthreads();
    float2 *dst = X1 + ((size_t)r * N + z) * N * H;
    for (int i = threadIdx.x; i < N * H; i += NT) dst[i] = P[i];
}

template <int N, int SRC>
__global__ void __launch_bounds__(PassA<N>::NT, SRC == SRC_TEX ? 2 : PassA<N>::MINB)
    passA_kernel(const float *__restrict__ rho, const float *__restrict__ rot9, float2 *__restrict__ X1,
                 cudaTextureObject_t tex, const int *__restrict__ box) {
    passA_body<N, SRC>(rho, rot9, X1, tex, box, blockIdx.x, blockIdx.y);
}

// ------------------------------------------------------- rotated resample
// rho2^R[r][z][y][x] = trilinear_periodic(rho2, R_r^T x_n) for a chunk of
// rotations.  No shared memory, so the whole L1 serves the gathers; each
// thread samples kZ nodes along z so that their loads are in flight together.
constexpr int kRsX = 32, kRsY = 8, kRsZ = 4;

// padded slices for the texture: slice z, local (x, y) in [0, N]^2, at
// slab[((z / SC)(N+1) + y) * pitch + (z % SC)(N+1) + x]
template <int N>
__global__ void pad_slices_kernel(const float *__restrict__ g, float *__restrict__ slab, size_t pitch_floats) {
    constexpr int SC = TexLayout<N>::SC;
    const size_t total = (size_t)N * (N + 1) * (N + 1);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % (N + 1));
        const size_t rest = i / (N + 1);
        const int y = (int)(rest % (N + 1)), z = (int)(rest / (N + 1));
        const size_t row = (size_t)(z / SC) * (N + 1) + y, col = (size_t)(z % SC) * (N + 1) + x;
        slab[row * pitch_floats + col] = __ldg(g + ((size_t)z * N + wrapN<N>(y)) * N + wrapN<N>(x));
    }
}

// Support of the moving density, pass 1: one CTA per z-slab, thread x walks
// column x.  Bit i of masks[8 a + i / 32] is set when the slab normal to axis
// a (0 = x, 1 = y, 2 = z) at index i holds a nonzero node (masks zeroed
// before the launch).
template <int N>
__global__ void __launch_bounds__(N) support_masks_kernel(const float *__restrict__ g, unsigned *__restrict__ masks) {
    constexpr int W = (N + 31) / 32;
    __shared__ unsigned ym[W];
    const int z = blockIdx.x, x = threadIdx.x, lane = x & 31;
    if (x < W) ym[x] = 0u;
    __syncthreads();
    const float *col = g + (size_t)z * N * N + x;
    bool nzc = false;
    for (int y = 0; y < N; ++y) {
        const bool nz = __ldg(col + (size_t)y * N) != 0.0f;
        nzc |= nz;
        if (__any_sync(0xffffffffu, nz) && lane == 0) atomicOr(&ym[y >> 5], 1u << (y & 31));
    }
    const unsigned xb = __ballot_sync(0xffffffffu, nzc);
    if (lane == 0 && xb) atomicOr(&masks[x >> 5], xb);
    const bool any = __syncthreads_or(nzc);
    if (x < W && ym[x]) atomicOr(&masks[8 + x], ym[x]);
    if (x == 0 && any) atomicOr(&masks[16 + (z >> 5)], 1u << (z & 31));
}

// Pass 2, one thread per axis: the nonzero slabs lie in the circular interval
// [lo, lo + len) that leaves out the longest circular run of zero slabs.  A
// cell with lower corner c touches it iff c is in [lo - 1, lo + len), stored
// as box[2a] = lo - 1 (mod N), box[2a + 1] = min(len + 1, N); an all-zero
// grid gives len 0 (no cell touches it).
template <int N>
__global__ void support_box_kernel(const unsigned *__restrict__ masks, int *__restrict__ box) {
    const int a = threadIdx.x;
    if (a >= 3) return;
    const unsigned *m = masks + 8 * a;
    auto bit = [m](int i) { return (m[i >> 5] >> (i & 31)) & 1u; };
    int first = -1;
    for (int i = 0; i < N && first < 0; ++i)
        if (bit(i)) first = i;
    int lo1 = 0, len1 = 0;
    if (first >= 0) {
        int best = 0, start = first, run = 0;  // longest zero run, and the set index after it
        for (int k = 1; k <= N; ++k) {
            const int i = (first + k) % N;
            if (bit(i)) {
                if (run > best) {
                    best = run;
                    start = i;
                }
                run = 0;
            } else {
                ++run;
            }
        }
        const int len = N - best;
        lo1 = (start - 1 + N) % N;
        len1 = len + 1 < N ? len + 1 : N;
    }
    box[2 * a] = lo1;
    box[2 * a + 1] = len1;
}

template <int N>
__global__ void __launch_bounds__(kRsX * kRsY) resample_chunk_kernel(const float *__restrict__ rho,
                                                                   const float *__restrict__ rot9,
                                                                   float *__restrict__ out) {
    const int tiles_x = N / kRsX, tiles_y = N / kRsY;
    int t = blockIdx.x;
    const int tx = t % tiles_x; t /= tiles_x;
    const int ty = t % tiles_y; t /= tiles_y;
    const int tz = t;
    const int r = blockIdx.y;
    float R[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) R[k] = __ldg(rot9 + 9 * r + k);
    const int x = tx * kRsX + (threadIdx.x % kRsX), y = ty * kRsY + (threadIdx.x / kRsX);
    const float cx = (float)(x - N / 2), cy = (float)(y - N / 2);
    const float ax = fmaf(R[0], cx, R[3] * cy), ay = fmaf(R[1], cx, R[4] * cy), az = fmaf(R[2], cx, R[5] * cy);
    float v[kRsZ];
#pragma unroll
    for (int j = 0; j < kRsZ; ++j) {
        const float cz = (float)(tz * kRsZ + j - N / 2);
        v[j] = trilinear_c<N>(rho, fmaf(R[6], cz, ax), fmaf(R[7], cz, ay), fmaf(R[8], cz, az));
    }
    float *o = out + (size_t)r * N * N * N + (size_t)y * N + x;
#pragma unroll
    for (int j = 0; j < kRsZ; ++j) o[(size_t)(tz * kRsZ + j) * N * N] = v[j];
}

// ------------------------------------------------------------------ pass B
// One CTA per CW consecutive columns f = ky* H + kx* (the flattened (ky, kx)
// index, contiguous in memory for every z) and rotation; all N z-values of
// a column.  Thread (c, g): column c < CW, digit group g < R2 (N = R1 R2).
// The z transforms keep their data in registers and use shared memory only
// for the three digit exchanges, each laid out [digit][digit][column] with
// the column fastest, so every shared access of a warp is one contiguous row:
//   forward  stage 1: thread (c, g) loads z = R2 n1 + g (n1 < R1) straight
//            from HBM, DFT-R1, twiddle W^(g k1), exchange;
//            stage 2: thread (c, k1) for k1 = g, g + R2, ...: DFT-R2 gives
//            slot s = R2 k1 + k2 (frequency k1 + R1 k2)
//   product  S = (h^3/N^3) rho1^ conj(rho2^R^), Gz = i pi kz~ S       Eqs. 5, 6a
//   inverse  stage 1 on the same registers (DFT-R2, conj twiddle), exchange;
//            stage 2: thread (c, g): DFT-R1 gives z = R2 n1 + g, stored
//            straight to HBM
// CWO != 0 selects another column-tile width (an autotuner candidate)
template <int N, int CWO = 0>
struct PassB {
    static constexpr int H = N / 2 + 1;
    static constexpr int R1 = Fact<N>::R1, R2 = Fact<N>::R2;
    static constexpr int CW = CWO ? CWO : (N >= 256 ? 16 : 32);  // columns per CTA (N H is a multiple)
    static constexpr int NT = CW * R2;
    static constexpr int KPT = (R1 + R2 - 1) / R2;      // stage-2 k1 values per thread
    static constexpr int MINB = CW < 32 && N < 256 ? 6 : (N >= 128 ? 3 : 4);
    static constexpr size_t smem = sizeof(float2) * (2 * (size_t)N * CW + N);
    static_assert((N * H) % CW == 0, "whole column tiles");
};

// Spectral-mode source of pass B: the table interpolated at os R^T k~, times
// (-1)^(kx+ky+kz) to move the phase back to the box corner; 0 on Nyquist
// planes.
// One rotated frequency read off the table: issue its four gathers (re and
// im at two slices) and keep the weights; spec_combine interpolates.  Split
// so that a thread keeps several samples' gathers in flight.
struct SpecTap {
    float4 ra, ia, rb, ib;
    float wx, wy, wz;
    bool zero, neg;
};
template <int N>
__device__ __forceinline__ SpecTap spec_issue(const SpecSrc &src, const float *R, int kx, int ky, int kz) {
    const int h = N / 2;
    SpecTap t;
    t.zero = kx == h || ky == h || kz == h;
    t.neg = ((kx + ky + kz) & 1) != 0;
    if (t.zero) return t;
    const float ks[3] = {(float)(src.os * (kx < h ? kx : kx - N)), (float)(src.os * (ky < h ? ky : ky - N)),
                         (float)(src.os * (kz < h ? kz : kz - N))};
    int i[3];
    float w[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) rot_coord(R[a], R[3 + a], R[6 + a], ks[0], ks[1], ks[2], i[a], w[a]);
    const int np = src.np, sc = src.sc;
    const int x0 = table_wrap(i[0], np), y0 = table_wrap(i[1], np);
    const int z0 = table_wrap(i[2], np), z1 = table_wrap(i[2] + 1, np);
    // one 2x2 gather per slice and component at the integer corner (x0+1,
    // y0+1) of the padded slice: w = (x0, y0), z = (x0+1, y0), x = (x0, y0+1),
    // y = (x0+1, y0+1); the wrapped neighbours come from the padding
    const float u0 = (float)((z0 % sc) * (np + 1) + x0) + 1.0f, v0 = (float)((z0 / sc) * (np + 1) + y0) + 1.0f;
    const float u1 = (float)((z1 % sc) * (np + 1) + x0) + 1.0f, v1 = (float)((z1 / sc) * (np + 1) + y0) + 1.0f;
    t.ra = tex2Dgather<float4>(src.tex, u0, v0, 0);
    t.ia = tex2Dgather<float4>(src.tex, u0, v0, 1);
    t.rb = tex2Dgather<float4>(src.tex, u1, v1, 0);
    t.ib = tex2Dgather<float4>(src.tex, u1, v1, 1);
    t.wx = w[0];
    t.wy = w[1];
    t.wz = w[2];
    return t;
}
__device__ __forceinline__ float2 spec_combine(const SpecTap &t) {
    if (t.zero) return make_float2(0.f, 0.f);
    const float2 a00 = make_float2(t.ra.w, t.ia.w), a01 = make_float2(t.ra.z, t.ia.z);
    const float2 a10 = make_float2(t.ra.x, t.ia.x), a11 = make_float2(t.ra.y, t.ia.y);
    const float2 b00 = make_float2(t.rb.w, t.ib.w), b01 = make_float2(t.rb.z, t.ib.z);
    const float2 b10 = make_float2(t.rb.x, t.ib.x), b11 = make_float2(t.rb.y, t.ib.y);
    auto lerp2 = [](float2 a, float2 b, float u) { return make_float2(fmaf(u, b.x - a.x, a.x), fmaf(u, b.y - a.y, a.y)); };
    const float2 v = lerp2(lerp2(lerp2(a00, a01, t.wx), lerp2(a10, a11, t.wx), t.wy),
                           lerp2(lerp2(b00, b01, t.wx), lerp2(b10, b11, t.wx), t.wy), t.wz);
    return t.neg ? make_float2(-v.x, -v.y) : v;
}
constexpr int kSpecInFlight = 4;  // samples whose gathers a thread issues together

// MODE 0: full middle pass (product, gradient, inverse z) -> Y1 = S', Y2 = Gz'
// MODE 1: forward only, spectrum * scale -> spec[kz*][ky*][kx*]  (stationary part)
// MODE 2: as MODE 0 with the rotated spectrum interpolated from a table
//         instead of transformed from resampled planes
// Loads of a pass's input intermediates: through the read-only path in a
// pass of its own (the producer was an earlier launch), at L2 (.cg) in the
// persistent kernel, where the producer is another block of the same launch
// and the non-coherent caches could hold an earlier chunk's lines.
template <bool COH>
__device__ __forceinline__ float2 ld_inter(const float2 *p) {
    if constexpr (COH) return __ldcg(p);
    else return __ldg(p);
}
template <bool COH>
__device__ __forceinline__ float2 ldg_inter(const float2 *p) {
    if constexpr (COH) return __ldcg(p);
    else return __ldg(p);
}

// The body of one pass B block: column tile bx of rotation r.
template <int N, int MODE, bool COH = false, int CWO = 0>
__device__ __forceinline__ void passB_body(const float2 *__restrict__ X1, const float2 *__restrict__ R1hat,
                                           float2 *__restrict__ Y1, float2 *__restrict__ Y2, float scale,
                                           const SpecSrc &spec, const float *__restrict__ rot9, unsigned bx,
                                           unsigned r) {
    __builtin_assume(bx < (1u << 24) && r < (1u << 16));  // the ranges of the blockIdx they stand for
    using PB = PassB<N, CWO>;
    constexpr int H = PB::H, R1 = PB::R1, R2 = PB::R2, CW = PB::CW, KPT = PB::KPT;
    constexpr size_t NH = (size_t)N * H;
    extern __shared__ __align__(16) float2 sm[];
    float2 *E = sm;                      // [k1][n2][c], later S's [n2][k1][c]
    float2 *G = sm + (size_t)N * CW;     // Gz's [n2][k1][c]
    float2 *twN = G + (size_t)N * CW;
    const int c = threadIdx.x % CW, g = threadIdx.x / CW;
    size_t f = (size_t)bx * CW + c;
    bool active = true;  // every column is live in modes 0 and 1
    load_tw<N>(twN);
    float2 X[KPT][R2];
    if constexpr (MODE == 2) {
        // a CTA takes CW consecutive frequencies kx (natural order, so that
        // neighbouring lanes read neighbouring table cells) of one ky slot;
        // the Nyquist column kx = N/2 is zero in this mode and is written by
        // the first tile of the row
        constexpr int HALF = N / 2, TILES = (HALF + CW - 1) / CW;
        const int kys = bx / TILES, tile = bx % TILES;
        const int kx = tile * CW + c;
        active = kx < HALF;
        f = (size_t)kys * H + (active ? xslot<N>(kx) : 0);
        if (tile == 0) {
            const size_t fq = (size_t)kys * H + HALF;
            for (int z = threadIdx.x; z < N; z += PB::NT) {
                Y1[(size_t)r * N * NH + (size_t)z * NH + fq] = make_float2(0.f, 0.f);
                Y2[(size_t)r * N * NH + (size_t)z * NH + fq] = make_float2(0.f, 0.f);
            }
        }
        float R[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) R[k] = __ldg(rot9 + 9 * r + k);
        const int ky = slot_freq<N>(kys);
        static_assert(R2 % kSpecInFlight == 0, "whole groups of samples");
#pragma unroll
        for (int j = 0; j < KPT; ++j) {
            const int k1 = g + R2 * j;
            if (k1 < R1) {
#pragma unroll
                for (int k0 = 0; k0 < R2; k0 += kSpecInFlight) {
                    SpecTap tap[kSpecInFlight];
#pragma unroll
                    for (int u = 0; u < kSpecInFlight; ++u)
                        if (active) tap[u] = spec_issue<N>(spec, R, kx, ky, slot_freq<N>(R2 * k1 + k0 + u));
#pragma unroll
                    for (int u = 0; u < kSpecInFlight; ++u)
                        X[j][k0 + u] = active ? spec_combine(tap[u]) : make_float2(0.f, 0.f);
                }
            }
        }
        __syncthreads();  // twiddles in place
    } else {
        // forward stage 1
        {
            float2 v[R1];
            const float2 *src = X1 + (size_t)r * N * NH + f;
#pragma unroll
            for (int n1 = 0; n1 < R1; ++n1) v[n1] = ld_inter<COH>(src + (size_t)(R2 * n1 + g) * NH);
            __syncthreads();  // twiddles in place
            RegDFT<R1, -1>::run(v);
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1)
                E[(k1 * R2 + g) * CW + c] = k1 ? cmul(v[k1], tw_pick<N, CW % 32 == 0>(twN, g * k1)) : v[k1];
        }
        __syncthreads();
        // forward stage 2: X[j][k2] = slot R2 k1 + k2 for k1 = g + R2 j
#pragma unroll
        for (int j = 0; j < KPT; ++j) {
            const int k1 = g + R2 * j;
            if (k1 < R1) {
#pragma unroll
                for (int n2 = 0; n2 < R2; ++n2) X[j][n2] = E[(k1 * R2 + n2) * CW + c];
                RegDFT<R2, -1>::run(X[j]);
            }
        }
    }
    if constexpr (MODE == 1) {
#pragma unroll
        for (int j = 0; j < KPT; ++j) {
            const int k1 = g + R2 * j;
            if (k1 < R1) {
#pragma unroll
                for (int k2 = 0; k2 < R2; ++k2) Y1[(size_t)(R2 * k1 + k2) * NH + f] = cscale(X[j][k2], scale);
            }
        }
        return;
    } else {
        if constexpr (MODE == 0) __syncthreads();  // E is free: it takes S's exchange
        // product, gradient, inverse stage 1
#pragma unroll
        for (int j = 0; j < KPT; ++j) {
            const int k1 = g + R2 * j;
            if (k1 < R1) {
                float2 Sv[R2], Gv[R2];
#pragma unroll
                for (int k2 = 0; k2 < R2; ++k2) {
                    const int s = R2 * k1 + k2;
                    const float2 a1 = active ? __ldg(R1hat + (size_t)s * NH + f) : make_float2(0.f, 0.f);
                    Sv[k2] = cmulc(a1, X[j][k2]);  // (h^3/N^3) rho1^ conj(rho2^R^)
                    Gv[k2] = cmul_is(Sv[k2], signed_k_mult<N>(slot_freq<N>(s)));
                }
                RegDFT<R2, +1>::run(Sv);
                RegDFT<R2, +1>::run(Gv);
#pragma unroll
                for (int n2 = 0; n2 < R2; ++n2) {
                    const float2 t = tw_pick<N, CW % 32 == 0>(twN, n2 * k1);
                    E[(n2 * R1 + k1) * CW + c] = n2 ? cmulc(Sv[n2], t) : Sv[n2];
                    G[(n2 * R1 + k1) * CW + c] = n2 ? cmulc(Gv[n2], t) : Gv[n2];
                }
            }
        }
        __syncthreads();
        // inverse stage 2: z = R2 n1 + g
        float2 v[R1];
        float2 *d1 = Y1 + (size_t)r * N * NH + f, *d2 = Y2 + (size_t)r * N * NH + f;
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) v[k1] = E[(g * R1 + k1) * CW + c];
        RegDFT<R1, +1>::run(v);
        if (active)
#pragma unroll
            for (int n1 = 0; n1 < R1; ++n1) d1[(size_t)(R2 * n1 + g) * NH] = v[n1];
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) v[k1] = G[(g * R1 + k1) * CW + c];
        RegDFT<R1, +1>::run(v);
        if (active)
#pragma unroll
            for (int n1 = 0; n1 < R1; ++n1) d2[(size_t)(R2 * n1 + g) * NH] = v[n1];
    }
}

template <int N, int MODE, int CWO = 0>
__global__ void __launch_bounds__(PassB<N, CWO>::NT, MODE == 2 ? 2 : PassB<N, CWO>::MINB) passB_kernel(const float2 *__restrict__ X1,
                                                                              const float2 *__restrict__ R1hat,
                                                                              float2 *__restrict__ Y1,
                                                                              float2 *__restrict__ Y2, float scale,
                                                                              SpecSrc spec,
                                                                              const float *__restrict__ rot9) {
    passB_body<N, MODE, false, CWO>(X1, R1hat, Y1, Y2, scale, spec, rot9, blockIdx.x, blockIdx.y);
}


// Torque spectra: the same forward z transform of X1 as pass B, then the
// three products Gm_a conj(rho2^R^) (a = x, y, z) with the stationary moment
// spectra and their inverse z transforms, straight to YT[a].
template <int N>
__global__ void __launch_bounds__(PassB<N>::NT, 2) passB_torque_kernel(const float2 *__restrict__ X1,
                                                                        const float2 *__restrict__ Gm,
                                                                        float2 *__restrict__ YT, size_t yt_stride) {
    constexpr int H = PassB<N>::H, R1 = PassB<N>::R1, R2 = PassB<N>::R2, CW = PassB<N>::CW,
                  KPT = PassB<N>::KPT;
    constexpr size_t NH = (size_t)N * H;
    extern __shared__ __align__(16) float2 sm[];
    float2 *E[3] = {sm, sm + (size_t)N * CW, sm + 2 * (size_t)N * CW};  // E[0] is also the forward exchange
    float2 *twN = sm + 3 * (size_t)N * CW;
    const int c = threadIdx.x % CW, g = threadIdx.x / CW;
    const size_t f = (size_t)blockIdx.x * CW + c;
    const int r = blockIdx.y;
    load_tw<N>(twN);
    {
        float2 v[R1];
        const float2 *src = X1 + (size_t)r * N * NH + f;
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) v[n1] = src[(size_t)(R2 * n1 + g) * NH];
        __syncthreads();
        RegDFT<R1, -1>::run(v);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1)
            E[0][(k1 * R2 + g) * CW + c] = k1 ? cmul(v[k1], tw_pick<N, CW % 32 == 0>(twN, g * k1)) : v[k1];
    }
    __syncthreads();
    float2 X[KPT][R2];
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
        const int k1 = g + R2 * j;
        if (k1 < R1) {
#pragma unroll
            for (int n2 = 0; n2 < R2; ++n2) X[j][n2] = E[0][(k1 * R2 + n2) * CW + c];
            RegDFT<R2, -1>::run(X[j]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
        const int k1 = g + R2 * j;
        if (k1 < R1) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                float2 T[R2];
#pragma unroll
                for (int k2 = 0; k2 < R2; ++k2)
                    T[k2] = cmulc(__ldg(Gm + (size_t)a * N * NH + (size_t)(R2 * k1 + k2) * NH + f), X[j][k2]);
                RegDFT<R2, +1>::run(T);
#pragma unroll
                for (int n2 = 0; n2 < R2; ++n2)
                    E[a][(n2 * R1 + k1) * CW + c] = n2 ? cmulc(T[n2], tw_pick<N, CW % 32 == 0>(twN, n2 * k1)) : T[n2];
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float2 v[R1];
        float2 *d = YT + a * yt_stride + (size_t)r * N * NH + f;
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) v[k1] = E[a][(g * R1 + k1) * CW + c];
        RegDFT<R1, +1>::run(v);
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) d[(size_t)(R2 * n1 + g) * NH] = v[n1];
    }
}

// ------------------------------------------------------------------ pass C
// One CTA per (z-plane, rotation) holding S'' and Gy'' side by side (pitch
// 2H+1), then Gz'' in place of S''.
// RBO / NTO != 0 select other rows per x batch / threads per CTA (autotuner
// candidates)
template <int N, int RBO = 0, int NTO = 0>
struct PassC {
    static constexpr int H = N / 2 + 1, HALF = N / 2;
    static constexpr int PW = H;  // plane pitch (odd): one half-spectrum plane at a time
    static constexpr int RB = RBO ? RBO : (N == 96) ? 48 : (N >= 64 ? 32 : 16);  // rows per x batch (divides N / 2)
    static_assert((N / 2) % RB == 0, "whole row batches");
    static constexpr int TP = N + 1;                                  // row-buffer pitch
    static constexpr int NT = NTO ? NTO : (N >= 128) ? 512 : (N >= 64 ? 256 : 128);
    static constexpr int MINB = (N >= 128) ? 2 : 1;
    static constexpr size_t smem = sizeof(float2) * ((size_t)N * PW + (size_t)RB * TP + N);
};

// Frequency k of the full x row, built from the half spectrum: k < N/2 reads
// xslot(k) as is, k > N/2 reads xslot(N-k) conjugated (Hermitian symmetry),
// k = N/2 reads the Nyquist slot; for the (E, Fx) row the value is also
// scaled by 1 + pi kx~ (kx~ = k, or k - N above N/2; 1 at the Nyquist
// frequency).
struct XEntry {
    int slot;
    float cs;    // +1, or -1 where the value is conjugated
    float mult;  // 1 + pi kx~
};

// The entries for all k = k1 + R1 K2 of one stage-1 item (k1 fixed,
// 0 <= k1 < R1; K2 compile-time).  With HALF = N/2 = a b (slot of m in a half
// row: b (m % a) + m / a) and a dividing R1, the slot is a per-item base plus a
// constant: t1 + (R1/a) K2 below N/2, t2 + (R1/a)(R2-K2-1) above it, where t1
// and t2 are the slots of k1 and of R1 - k1; only the Nyquist frequency
// (K2 = R2/2, k1 = 0) is special.  kx~ is formed as k1 + R1 K2 (- N) in exact
// small-integer float arithmetic.
template <int N, int R1>
struct XItem {
    static constexpr int R2 = N / R1, HALF = N / 2, A = Fact<N / 2>::R1, B = Fact<N / 2>::R2;
    static_assert(R1 % A == 0, "the half row's first digit divides the x pass's");
    int t1, t2;
    float k1f;
    bool nyq;  // k1 = 0: K2 = R2/2 is the Nyquist frequency
    __device__ __forceinline__ explicit XItem(int k1) {
        const int j = R1 - k1;
        t1 = B * (k1 % A) + k1 / A;
        t2 = B * (j % A) + j / A;
        k1f = (float)k1;
        nyq = k1 == 0;
    }
    template <int K2>
    __device__ __forceinline__ XEntry entry() const {
        XEntry e;
        if constexpr (2 * K2 < R2) {
            e.slot = t1 + (R1 / A) * K2;
            e.cs = 1.0f;
            e.mult = 1.0f + kPi * (k1f + (float)(R1 * K2));
        } else {
            e.slot = t2 + (R1 / A) * (R2 - K2 - 1);
            e.cs = -1.0f;
            e.mult = 1.0f + kPi * (k1f + (float)(R1 * K2 - N));
            if constexpr (2 * K2 == R2) {
                if (nyq) {
                    e.slot = HALF;
                    e.cs = 1.0f;
                    e.mult = 1.0f;
                }
            }
        }
        return e;
    }
};

// One complex inverse DFT of length N per row, input built from half-spectrum
// rows (pitch PW) by Hermitian symmetry; real part -> out0, imaginary -> out1.
// PAIR 0: Z[k] = A(k) (1 + pi kx~)         -> (E, Fx) when A = S''
// PAIR 1: Z[k] = -(B(k) + i A(k))          -> two real fields, -IDFT(B) and
//         -IDFT(A), from two rows (of one field or of two)
// Row j of A at planeA + j PW + colA, of B at planeB + j PW + colB; rows
// [0, ROWS) go to output rows [0, ROWS), RB rows per batch through the row
// buffer Tb (pitch TP).
// Torque epilogue of an x pass (analytic torque): the stored value is
// -(IDFT) of the pass minus (t x F)_axis at the lag, i.e. T = C(G, rho2R) -
// t x F; F is this plane's force, already written by the same CTA.
struct TorqueCorr {
    const float *F[3];  // row y of F_d at F[d] + y N
    int axis;
    int zlag;           // signed z lag of the plane
    int row1;           // out1's rows are out0's rows + row1
};

// store with an L2 evict-last policy: rows that the same CTA reads back soon
__device__ __forceinline__ uint64_t l2_keep_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void st_keep(float *p, float v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol) : "memory");
}

// x_pass calls hook(y0) once per row batch, right after the barrier that ends
// the batch's reads of the plane (the rows it read may then be overwritten)
struct NoHook {
    __device__ __forceinline__ void operator()(int) const {}
};

template <int N, int PAIR, int PW, int RB, int TP, int NT, int ROWS, bool CTW = true, bool KEEP0 = false,
          bool KEEP1 = false, class Hook = NoHook, int XR1 = 0>
__device__ __forceinline__ void x_pass(const float2 *planeA, const float2 *planeB, int colA, int colB,
                                       float2 *Tb, const float2 *twN,
                                       float *__restrict__ out0, float *__restrict__ out1,
                                       const TorqueCorr *tc = nullptr, const Hook &hook = Hook()) {
    // N = R1 R2, by default with the longer digit second, so that stage 2
    // runs with lanes along it: its reads of the row buffer are contiguous and
    // its outputs (x = R2 n1 + n2) go straight to HBM as full 32-byte sectors;
    // XR1 picks the first digit instead (the autotuner's radix candidate)
    constexpr int R1 = XR1 ? XR1 : (Fact<N>::R1 < Fact<N>::R2 ? Fact<N>::R1 : Fact<N>::R2);
    constexpr int R2 = N / R1;
    static_assert(N % R1 == 0 && R2 >= 8, "whole digits; stage 2 writes at least 32-byte runs");
#pragma unroll 1
    for (int y0 = 0; y0 < ROWS; y0 += RB) {
        // stage 1 (inverse), items (row, k1): Tb[row][R2 k1 + n2] from Z[k1 + R1 k2]
#pragma unroll 1
        for (int w = threadIdx.x; w < RB * R1; w += NT) {
            const int row = w % RB, k1 = w / RB;
            const float2 *pa = planeA + (size_t)(y0 + row) * PW + colA;
            const float2 *pb = planeB + (size_t)(y0 + row) * PW + colB;
            float2 v[R2];
            const XItem<N, R1> xi(k1);
            static_for<0, R2>([&](auto kk) {
                constexpr int k2 = decltype(kk)::value;
                const XEntry e = xi.template entry<k2>();
                if constexpr (PAIR == 0) {
                    const float2 a = pa[e.slot];
                    v[k2] = make_float2(e.mult * a.x, (e.mult * e.cs) * a.y);
                } else {
                    const float2 gy = pb[e.slot], gz = pa[e.slot];
                    v[k2] = make_float2(fmaf(e.cs, gz.y, -gy.x), fmaf(-e.cs, gy.y, -gz.x));  // -(gy + i gz)
                }
            });
            RegDFT<R2, +1>::run(v);
            float2 *tr = Tb + row * TP + R2 * k1;
#pragma unroll
            for (int n2 = 0; n2 < R2; ++n2) {
                // twiddles from constant memory where k1 is warp-uniform (RB a
                // multiple of 32), else from the shared table
                const float2 t = (CTW && RB % 32 == 0) ? tw_uniform<N>(n2 * k1) : twN[n2 * k1];
                tr[n2] = n2 ? cmulc(v[n2], t) : v[n2];
            }
        }
        __syncthreads();
        hook(y0);
        // stage 2 (inverse), items (row, n2), lanes along n2: x = R2 n1 + n2
#pragma unroll 1
        for (int w = threadIdx.x; w < RB * R2; w += NT) {
            const int n2 = w % R2, row = w / R2;
            const float2 *tr = Tb + row * TP + n2;
            float2 v[R1];
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1) v[k1] = tr[R2 * k1];
            RegDFT<R1, +1>::run(v);
            const int y = y0 + row;
            const size_t o = (size_t)y * N + n2;
            if (tc) {
                const float h = 2.0f / N, tz = tc->zlag * h;
                auto sgn = [](int j) { return j < N / 2 ? j : j - N; };
                const float ty0 = sgn(y) * h, ty1 = sgn(y + tc->row1) * h;
#pragma unroll
                for (int n1 = 0; n1 < R1; ++n1) {
                    const int x = R2 * n1 + n2;
                    const size_t oo = o + (size_t)R2 * n1, o1 = oo + (size_t)tc->row1 * N;
                    const float tx = sgn(x) * h;
                    const float f0[3] = {tc->F[0][oo], tc->F[1][oo], tc->F[2][oo]};
                    const float f1[3] = {tc->F[0][o1], tc->F[1][o1], tc->F[2][o1]};
                    float c0, c1;
                    if (tc->axis == 0) {
                        c0 = ty0 * f0[2] - tz * f0[1];
                        c1 = ty1 * f1[2] - tz * f1[1];
                    } else if (tc->axis == 1) {
                        c0 = tz * f0[0] - tx * f0[2];
                        c1 = tz * f1[0] - tx * f1[2];
                    } else {
                        c0 = tx * f0[1] - ty0 * f0[0];
                        c1 = tx * f1[1] - ty1 * f1[0];
                    }
                    out0[oo] = -v[n1].x - c0;
                    out1[oo] = -v[n1].y - c1;
                }
            } else {
                uint64_t pol = 0;
                if constexpr (KEEP0 || KEEP1) pol = l2_keep_policy();
#pragma unroll
                for (int n1 = 0; n1 < R1; ++n1) {
                    if constexpr (KEEP0)
                        st_keep(out0 + o + (size_t)R2 * n1, v[n1].x, pol);
                    else
                        out0[o + (size_t)R2 * n1] = v[n1].x;
                    if constexpr (KEEP1)
                        st_keep(out1 + o + (size_t)R2 * n1, v[n1].y, pol);
                    else
                        out1[o + (size_t)R2 * n1] = v[n1].y;
                }
            }
        }
        __syncthreads();
    }
}

// The y inverse after stage 1 (its barrier included): the Nyquist column's
// two steps and stage 2, in place in the plane
template <int N, int NT>
__device__ __forceinline__ void y_inverse_tail(float2 *plane, const float2 *twN) {
    constexpr int HALF = N / 2, R1 = Fact<N>::R1, R2 = Fact<N>::R2, PW = PassC<N>::PW;
    // Nyquist column, step 1 (warp 0, items k1, in place): slots R2 k1 + k2
    if (threadIdx.x < R1) {
        const int k1 = threadIdx.x;
        float2 *p = plane + (size_t)(R2 * k1) * PW + HALF;
        float2 v[R2];
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) v[k2] = p[k2 * PW];
        RegDFT<R2, +1>::run(v);
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) p[n2 * PW] = n2 ? cmulc(v[n2], twN[n2 * k1]) : v[n2];
    }
    // stage 2: items (c, n2); every item is read before any row is written
    constexpr int ITEMS = HALF * R2, IPT = (ITEMS + NT - 1) / NT;
    float2 v[IPT][R1];
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
        const int w = threadIdx.x + j * NT;
        if (w < ITEMS) {
            const int c = w % HALF, n2 = w / HALF;
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1) v[j][k1] = plane[(n2 * R1 + k1) * PW + c];
            RegDFT<R1, +1>::run(v[j]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
        const int w = threadIdx.x + j * NT;
        if (w < ITEMS) {
            const int c = w % HALF, n2 = w / HALF;
#pragma unroll
            for (int n1 = 0; n1 < R1; ++n1) plane[(R2 * n1 + n2) * PW + c] = v[j][n1];
        }
    }
    // Nyquist column, step 2 (warp 1, items n2, in place): natural y = R2 n1 + n2
    if (threadIdx.x >= 32 && threadIdx.x < 32 + R2) {
        const int n2 = threadIdx.x - 32;
        float2 *p = plane + (size_t)n2 * PW + HALF;
        float2 u[R1];
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) u[k1] = p[k1 * R2 * PW];
        RegDFT<R1, +1>::run(u);
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) p[n1 * R2 * PW] = u[n1];
    }
    __syncthreads();
}

// Inverse y transform of one z-plane's H half-spectrum columns: global rows
// src[s H + c] (ky slot order) -> plane[y PW + c] (natural y).  The N/2 main
// columns run register-centric (stage 1 straight from HBM, the digit
// exchange through the plane buffer as [n2][k1][c], stage 2 back into the
// plane's rows).  The Nyquist column is loaded while stage 1 runs and
// transformed in place in two small steps that ride along with stage 2's
// read and write phases (one warp each), so it costs no barrier of its own.
// MUL multiplies input row s by i pi ky~(s) on the way in (forms Gy from S').
template <int N, bool MUL, bool CTW = true, int NT = PassC<N>::NT, bool COH = false, int YU = 1>
__device__ __forceinline__ void y_inverse_plane(const float2 *__restrict__ src, float2 *plane, const float2 *twN) {
    constexpr int H = N / 2 + 1, HALF = N / 2, R1 = Fact<N>::R1, R2 = Fact<N>::R2, PW = PassC<N>::PW;
    static_assert(NT >= N && NT >= 32 + R2, "one Nyquist value per thread; Nyquist steps on warps 0 and 1");
    float2 nyq = make_float2(0.f, 0.f);
    if (threadIdx.x < N) nyq = ldg_inter<COH>(src + (size_t)threadIdx.x * H + HALF);
    // stage 1: items (c, k1), slots R2 k1 + k2; YU items' loads in flight per thread
#pragma unroll 1
    for (int w0 = threadIdx.x; w0 < HALF * R1; w0 += NT * YU) {
        float2 v[YU][R2];
#pragma unroll
        for (int u = 0; u < YU; ++u) {
            const int w = w0 + u * NT;
            if ((HALF * R1) % (NT * YU) == 0 || w < HALF * R1) {
                const int c = w % HALF, k1 = w / HALF;
#pragma unroll
                for (int k2 = 0; k2 < R2; ++k2) v[u][k2] = ldg_inter<COH>(src + (size_t)(R2 * k1 + k2) * H + c);
            }
        }
#pragma unroll
        for (int u = 0; u < YU; ++u) {
            const int w = w0 + u * NT;
            if ((HALF * R1) % (NT * YU) == 0 || w < HALF * R1) {
                const int c = w % HALF, k1 = w / HALF;
                if constexpr (MUL) {
#pragma unroll
                    for (int k2 = 0; k2 < R2; ++k2)
                        v[u][k2] = cmul_is(v[u][k2], signed_k_mult<N>(slot_freq<N>(R2 * k1 + k2)));
                }
                RegDFT<R2, +1>::run(v[u]);
#pragma unroll
                for (int n2 = 0; n2 < R2; ++n2) {
                    // k1 is warp-uniform when N/2 is a multiple of 32
                    const float2 t = (CTW && HALF % 32 == 0) ? tw_uniform<N>(n2 * k1) : twN[n2 * k1];
                    plane[(n2 * R1 + k1) * PW + c] = n2 ? cmulc(v[u][n2], t) : v[u][n2];
                }
            }
        }
    }
    if (threadIdx.x < N) {
        if constexpr (MUL) nyq = cmul_is(nyq, signed_k_mult<N>(slot_freq<N>(threadIdx.x)));
        plane[threadIdx.x * PW + HALF] = nyq;
    }
    __syncthreads();
    y_inverse_tail<N, NT>(plane, twN);
}

// The same inverse on a plane that bulk copies bring into shared memory
// (plane[s PW + c] = src[s H + c], arriving on mbar's phase `parity`):
// stage 1 reads its items from the plane into registers, and after a barrier
// writes them back in place.
template <int N, bool MUL, bool CTW, int NT>
__device__ __forceinline__ void y_inverse_plane_smem(float2 *plane, const float2 *twN, unsigned long long *mbar,
                                                     unsigned parity) {
    constexpr int HALF = N / 2, R1 = Fact<N>::R1, R2 = Fact<N>::R2, PW = PassC<N>::PW;
    static_assert(PW == N / 2 + 1, "the plane's rows are the source rows");
    static_assert(NT >= N && NT >= 32 + R2, "one Nyquist value per thread; Nyquist steps on warps 0 and 1");
    constexpr int ITEMS = HALF * R1, IPT = (ITEMS + NT - 1) / NT;
    mbar_wait_bounded(mbar, parity);
    float2 v[IPT][R2];
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
        const int w = threadIdx.x + j * NT;
        if (ITEMS % NT == 0 || w < ITEMS) {
            const int c = w % HALF, k1 = w / HALF;
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) {
                v[j][k2] = plane[(R2 * k1 + k2) * PW + c];
                if constexpr (MUL) v[j][k2] = cmul_is(v[j][k2], signed_k_mult<N>(slot_freq<N>(R2 * k1 + k2)));
            }
            RegDFT<R2, +1>::run(v[j]);
        }
    }
    if constexpr (MUL) {
        if (threadIdx.x < N) {  // the Nyquist column: no stage-1 item touches it
            float2 *q = plane + (size_t)threadIdx.x * PW + HALF;
            *q = cmul_is(*q, signed_k_mult<N>(slot_freq<N>(threadIdx.x)));
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
        const int w = threadIdx.x + j * NT;
        if (ITEMS % NT == 0 || w < ITEMS) {
            const int c = w % HALF, k1 = w / HALF;
#pragma unroll
            for (int n2 = 0; n2 < R2; ++n2) {
                const float2 t = (CTW && HALF % 32 == 0) ? tw_uniform<N>(n2 * k1) : twN[n2 * k1];
                plane[(n2 * R1 + k1) * PW + c] = n2 ? cmulc(v[j][n2], t) : v[j][n2];
            }
        }
    }
    __syncthreads();
    y_inverse_tail<N, NT>(plane, twN);
}

// Pass C holds one half-spectrum plane at a time (about 100 KB of shared
// memory at 128^3, two CTAs per SM):
//   S'  -> y inverse -> rows of S'' (1 + pi kx~)      -> E + i Fx
//   S'  (again, from L2) times i pi ky~ = Gy -> y inverse -> rows p and
//       p + N/2 paired in one complex x inverse    -> Fy
//   Gz' -> y inverse -> rows paired likewise          -> Fz
// The body of one pass C block: plane z of rotation r.  NT threads (the
// kernel's 512 at N = 128, a persistent block's 256); COH as for ld_inter.
// L2 prefetch of `bytes` (a multiple of 16, 16-byte aligned) at p
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// x_pass hook of the bulk-staged pass C: once a row batch of the plane has
// been read, thread 0 starts the copies of the same rows of the next plane
// (`src`; ROWSETS 2: the batch read rows y0.. and N/2 + y0..); the first
// batch opens the mbarrier phase for the whole plane
template <int N, int RB, int ROWSETS>
struct RowRefill {
    float2 *plane;
    const float2 *src;
    unsigned long long *mbar;
    __device__ __forceinline__ void operator()(int y0) const {
        constexpr int H = N / 2 + 1;
        constexpr unsigned BYTES = sizeof(float2) * RB * H;
        static_assert(BYTES % 16 == 0 && (sizeof(float2) * H * RB) % 16 == 0, "16-byte copies");
        if (threadIdx.x != 0) return;
        fence_proxy_async_smem();
        if (y0 == 0) mbar_expect(mbar, (unsigned)(sizeof(float2) * N * H));
        bulk_g2s(plane + (size_t)y0 * H, src + (size_t)y0 * H, BYTES, mbar);
        if constexpr (ROWSETS == 2) bulk_g2s(plane + (size_t)(N / 2 + y0) * H, src + (size_t)(N / 2 + y0) * H, BYTES, mbar);
    }
};

// YU: y-stage items whose loads a thread keeps in flight; PF: prefetch the
// block's Gz' plane into L2 when the block starts (it is read third); BK:
// bring each input plane into shared memory by bulk copies, the next plane's
// rows issued as the x pass frees them (one mbarrier, one phase per plane)
template <int N, bool TQ, int NT = PassC<N>::NT, bool COH = false, int RBO = 0, int YU = 1, bool PF = false,
          bool BK = false, int XR1 = 0>
__device__ __forceinline__ void passC_body(const float2 *__restrict__ Y1, const float2 *__restrict__ Y2,
                                           const FieldPtrs &out, const float2 *__restrict__ YT, size_t yt_stride,
                                           unsigned zu, unsigned ru) {
    __builtin_assume(zu < (1u << 16) && ru < (1u << 16));  // the ranges of the blockIdx they stand for
    const int z = (int)zu, r = (int)ru;
    using PC = PassC<N, RBO>;
    constexpr int H = PC::H, PW = PC::PW, RB = PC::RB, TP = PC::TP, HALF = N / 2;
    extern __shared__ __align__(16) float2 sm[];
    float2 *plane = sm;                       // [N][PW]
    float2 *Tb = plane + (size_t)N * PW;      // [RB][TP]
    float2 *twN = Tb + (size_t)RB * TP;
    const float2 *s1 = Y1 + ((size_t)r * N + z) * N * H;
    const size_t fo = (size_t)r * out.rot_stride + (size_t)z * N * N;
    if constexpr (BK) {
        // (inside the one-launch queue, COH: the thread that issues the copies
        // has acquired the producers' release and fenced the async proxy)
        static_assert(!TQ && YU == 1 && !PF, "the bulk-staged form of the E/F kernel");
        static_assert((sizeof(float2) * N * H) % 16 == 0, "whole 16-byte units");
        // the mbarrier sits after the twiddles (8-byte aligned)
        unsigned long long *mbar = reinterpret_cast<unsigned long long *>(twN + N);
        const float2 *s2 = Y2 + ((size_t)r * N + z) * N * H;
        if (threadIdx.x == 0) {
            mbar_init1(mbar);
            mbar_expect(mbar, (unsigned)(sizeof(float2) * N * H));
            bulk_g2s(plane, s1, (unsigned)(sizeof(float2) * N * H), mbar);
        }
        load_tw<N>(twN);
        __syncthreads();
        // E + i Fx; its batches refill the plane with S' (for Gy)
        y_inverse_plane_smem<N, false, true, NT>(plane, twN, mbar, 0);
        x_pass<N, 0, PW, RB, TP, NT, N, true, false, false, RowRefill<N, RB, 1>, XR1>(
            plane, plane, 0, 0, Tb, twN, out.E + fo, out.Fx + fo, nullptr, RowRefill<N, RB, 1>{plane, s1, mbar});
        // Fy; its batches refill the plane with Gz'
        y_inverse_plane_smem<N, true, true, NT>(plane, twN, mbar, 1);
        x_pass<N, 1, PW, RB, TP, NT, HALF, true, false, false, RowRefill<N, RB, 2>, XR1>(
            plane + (size_t)HALF * PW, plane, 0, 0, Tb, twN, out.Fy + fo, out.Fy + fo + (size_t)HALF * N, nullptr,
            RowRefill<N, RB, 2>{plane, s2, mbar});
        // Fz
        y_inverse_plane_smem<N, false, true, NT>(plane, twN, mbar, 0);
        x_pass<N, 1, PW, RB, TP, NT, HALF, true, false, false, NoHook, XR1>(
            plane + (size_t)HALF * PW, plane, 0, 0, Tb, twN, out.Fz + fo, out.Fz + fo + (size_t)HALF * N);
        return;
    }
    if constexpr (PF) {
        static_assert((sizeof(float2) * N * H) % 16 == 0, "whole 16-byte units");
        if (threadIdx.x == 0) prefetch_l2(Y2 + ((size_t)r * N + z) * N * H, (unsigned)(sizeof(float2) * N * H));
    }
    load_tw<N>(twN);
    __syncthreads();
    // E + i Fx
    y_inverse_plane<N, false, !TQ, NT, COH, YU>(s1, plane, twN);
    // with the torque phases (TQ) this CTA reads its force rows back: keep them in L2
    x_pass<N, 0, PW, RB, TP, NT, N, !TQ, false, TQ>(plane, plane, 0, 0, Tb, twN, out.E + fo, out.Fx + fo);
    // Fy from Gy = i pi ky~ S'
    y_inverse_plane<N, true, !TQ, NT, COH, YU>(s1, plane, twN);
    x_pass<N, 1, PW, RB, TP, NT, HALF, !TQ, TQ, TQ>(plane + (size_t)HALF * PW, plane, 0, 0, Tb, twN, out.Fy + fo,
                                      out.Fy + fo + (size_t)HALF * N);
    // Fz
    y_inverse_plane<N, false, !TQ, NT, COH, YU>(Y2 + ((size_t)r * N + z) * N * H, plane, twN);
    x_pass<N, 1, PW, RB, TP, NT, HALF, !TQ, TQ, TQ>(plane + (size_t)HALF * PW, plane, 0, 0, Tb, twN, out.Fz + fo,
                                      out.Fz + fo + (size_t)HALF * N);
    if constexpr (TQ) {
        // analytic torque: T_a = C(G_a, rho2R) - (t x F)_a, rows paired like Fy
        float *T[3] = {out.Tx, out.Ty, out.Tz};
#pragma unroll 1
        for (int a = 0; a < 3; ++a) {
            y_inverse_plane<N, false, !TQ, NT, COH>(YT + a * yt_stride + ((size_t)r * N + z) * N * H, plane, twN);
            const TorqueCorr tc{{out.Fx + fo, out.Fy + fo, out.Fz + fo}, a, z < HALF ? z : z - N, HALF};
            x_pass<N, 1, PW, RB, TP, NT, HALF, !TQ>(plane + (size_t)HALF * PW, plane, 0, 0, Tb, twN, T[a] + fo,
                                              T[a] + fo + (size_t)HALF * N, &tc);
        }
    }
}

template <int N, bool TQ, int RBO = 0, int NTO = 0, int YU = 1, bool PF = false, bool BK = false, int XR1 = 0>
__global__ void __launch_bounds__(PassC<N, RBO, NTO>::NT, PassC<N, RBO, NTO>::MINB) passC_kernel(const float2 *__restrict__ Y1,
                                                                              const float2 *__restrict__ Y2,
                                                                              FieldPtrs out,
                                                                              const float2 *__restrict__ YT,
                                                                              size_t yt_stride) {
    passC_body<N, TQ, PassC<N, RBO, NTO>::NT, false, RBO, YU, PF, BK, XR1>(Y1, Y2, out, YT, yt_stride, blockIdx.x,
                                                                           blockIdx.y);
}
// dynamic shared memory of the bulk-staged form: the mbarrier after the twiddles
template <int N, int RBO = 0, int NTO = 0>
constexpr size_t passC_bulk_smem() {
    return PassC<N, RBO, NTO>::smem + 16;
}

// the stationary moment fields G_a = (u x F)_a / h^3 (F = -h^3 grad rho1)
template <int N>
__global__ void moment_fields_kernel(const float *__restrict__ Fx, const float *__restrict__ Fy,
                                     const float *__restrict__ Fz, float *__restrict__ G) {
    const size_t n3 = (size_t)N * N * N;
    const float h = 2.0f / N, inv_h3 = 1.0f / (h * h * h);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n3; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % N), y = (int)((i / N) % N), z = (int)(i / ((size_t)N * N));
        const float ux = -1.0f + x * h, uy = -1.0f + y * h, uz = -1.0f + z * h;
        const float fx = Fx[i], fy = Fy[i], fz = Fz[i];
        G[i] = (uy * fz - uz * fy) * inv_h3;
        G[n3 + i] = (uz * fx - ux * fz) * inv_h3;
        G[2 * n3 + i] = (ux * fy - uy * fx) * inv_h3;
    }
}

// ------------------------------------------------------- pencil pipeline
// For grids whose planes do not fit one CTA's shared memory (N = 256): the
// x and y stages of passes A and C run as separate row-batch and column-chunk
// kernels with the intermediates in global memory (same layouts and slot
// orders as the slab passes, so pass B is shared).
template <int N>
struct Pencil {
    static constexpr int H = N / 2 + 1, HALF = N / 2;
    static constexpr int RBX = 16;                      // rows per CTA, x stages
    static constexpr int CY = 16;                       // kx columns per CTA, y stages
    static constexpr int NCY = (H + CY - 1) / CY;
    static constexpr int NT = 256;
    // texture x forward: 4 samples in flight per thread and 4 CTAs per SM (64
    // registers) beat 8 in flight at 2 CTAs per SM; 96 would spill at 64
    static constexpr int XU = 4, XMINB = (N & (N - 1)) == 0 ? 4 : 1;
    static constexpr int PW = 3 * H;                    // x-inverse row pitch: S | Gy | Gz (odd)
    static constexpr int TP = N + 1;
    static constexpr size_t smem_xfwd = sizeof(float2) * ((size_t)RBX * H + N + HALF);
    static constexpr size_t smem_yfwd = sizeof(float2) * ((size_t)N * CY + N);
    static constexpr size_t smem_yinv = sizeof(float2) * ((size_t)N * 3 * CY + N);
    static constexpr size_t smem_xinv =
        sizeof(float2) * ((size_t)RBX * PW + (size_t)RBX * TP + N);
};

// x forward: RBX rows (q = z N + y) of rotation r -> half-spectrum rows Xa[r][q][kx*].
// TEX: the rows are sampled from the moving part's texture at the rotated
// node positions (the resample fused in, the same samples bit for bit as
// pass A's) instead of read from resampled planes.
template <int N, bool TEX>
__global__ void __launch_bounds__(Pencil<N>::NT, Pencil<N>::XMINB) xfwd_kernel(const float *__restrict__ planes,
                                                             float2 *__restrict__ Xa, cudaTextureObject_t tex,
                                                             const float *__restrict__ rot9,
                                                             const int *__restrict__ box) {
    constexpr int H = Pencil<N>::H, HALF = Pencil<N>::HALF, RBX = Pencil<N>::RBX, NT = Pencil<N>::NT;
    extern __shared__ __align__(16) float2 sm[];
    float2 *P = sm;               // [RBX][H]
    float2 *twN = P + RBX * H;
    float2 *twH = twN + N;
    const size_t q0 = (size_t)blockIdx.x * RBX;
    const int r = blockIdx.y;
    if constexpr (TEX) {
        float R[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) R[k] = __ldg(rot9 + 9 * r + k);
        float *Pf = reinterpret_cast<float *>(P);
        static_assert(N % RBX == 0, "a CTA's rows lie in one z-slice");
        tex_resample<N, NT, RBX, false, Pencil<N>::XU>(tex, R, Pf, box, (int)(q0 % N), (int)(q0 / N));
        load_tw<N>(twN);
        load_tw<HALF>(twH);
    } else {
        const float2 *src = reinterpret_cast<const float2 *>(planes + ((size_t)r * N * N + q0) * N);
        for (int i = threadIdx.x; i < RBX * HALF; i += NT) {
            const int row = i / HALF, x2 = i % HALF;
            cp_async8(P + row * H + x2, src + i);
        }
        load_tw<N>(twN);
        load_tw<HALF>(twH);
        cp_async_wait_all();
    }
    __syncthreads();
    fft_lines<HALF, -1, RBX, 1, H, NT>(P, twH);
    for (int i = threadIdx.x; i < RBX * (N / 4 + 1); i += NT) {
        const int y = i % RBX, k = i / RBX;
        float2 *row = P + y * H;
        if (k == 0) {
            const float2 z0 = row[0];
            row[0] = make_float2(z0.x + z0.y, 0.f);
            row[HALF] = make_float2(z0.x - z0.y, 0.f);
        } else if (4 * k == N) {
            const int sl = perm_slot<HALF>(k);
            row[sl] = cconj(row[sl]);
        } else {
            const int s1 = perm_slot<HALF>(k), s2 = perm_slot<HALF>(HALF - k);
            const float2 a = row[s1], b = row[s2];
            const float2 Ek = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
            const float2 Ok = make_float2(0.5f * (a.y + b.y), -0.5f * (a.x - b.x));
            const float2 WO = cmul(twN[k], Ok);
            row[s1] = cadd(Ek, WO);
            row[s2] = cconj(csub(Ek, WO));
        }
    }
    __syncthreads();
    float2 *dst = Xa + ((size_t)r * N * N + q0) * H;
    for (int i = threadIdx.x; i < RBX * H; i += NT) dst[i] = P[i];
}

// y forward: kx columns [c0, c0 + CY) of plane z -> X1[r][z][ky*][kx*]
template <int N>
__global__ void __launch_bounds__(Pencil<N>::NT) yfwd_kernel(const float2 *__restrict__ Xa,
                                                             float2 *__restrict__ X1) {
    constexpr int H = Pencil<N>::H, CY = Pencil<N>::CY, NCY = Pencil<N>::NCY, NT = Pencil<N>::NT;
    extern __shared__ __align__(16) float2 sm[];
    float2 *T = sm;               // [N][CY]
    float2 *twN = T + N * CY;
    const int z = blockIdx.x / NCY, c0 = (blockIdx.x % NCY) * CY, r = blockIdx.y;
    const int cw = min(CY, H - c0);
    const float2 *src = Xa + ((size_t)r * N + z) * N * H + c0;
    for (int i = threadIdx.x; i < N * CY; i += NT) {
        const int y = i / CY, c = i % CY;
        if (c < cw) cp_async8(T + i, src + (size_t)y * H + c);
        else T[i] = make_float2(0.f, 0.f);
    }
    load_tw<N>(twN);
    cp_async_wait_all();
    __syncthreads();
    fft_lines<N, -1, CY, CY, 1, NT>(T, twN);
    float2 *dst = X1 + ((size_t)r * N + z) * N * H + c0;
    for (int i = threadIdx.x; i < N * CY; i += NT) {
        const int sl = i / CY, c = i % CY;
        if (c < cw) dst[(size_t)sl * H + c] = T[i];
    }
}

// y inverse of S', Gy = i pi ky~ S' and Gz' for kx columns [c0, c0 + CY) of plane z
template <int N>
__global__ void __launch_bounds__(Pencil<N>::NT) yinv_kernel(const float2 *__restrict__ Y1,
                                                             const float2 *__restrict__ Y2,
                                                             float2 *__restrict__ ZS, float2 *__restrict__ ZGy,
                                                             float2 *__restrict__ ZGz) {
    constexpr int H = Pencil<N>::H, CY = Pencil<N>::CY, NCY = Pencil<N>::NCY, NT = Pencil<N>::NT,
                  W3 = 3 * CY;
    extern __shared__ __align__(16) float2 sm[];
    float2 *T = sm;               // [N][3 CY]: S | Gy | Gz
    float2 *twN = T + N * W3;
    const int z = blockIdx.x / NCY, c0 = (blockIdx.x % NCY) * CY, r = blockIdx.y;
    const int cw = min(CY, H - c0);
    const size_t base = ((size_t)r * N + z) * N * H + c0;
    for (int i = threadIdx.x; i < N * CY; i += NT) {
        const int sl = i / CY, c = i % CY;
        if (c < cw) {
            cp_async8(T + sl * W3 + c, Y1 + base + (size_t)sl * H + c);
            cp_async8(T + sl * W3 + 2 * CY + c, Y2 + base + (size_t)sl * H + c);
        } else {
            T[sl * W3 + c] = make_float2(0.f, 0.f);
            T[sl * W3 + 2 * CY + c] = make_float2(0.f, 0.f);
        }
    }
    load_tw<N>(twN);
    cp_async_wait_all();
    __syncthreads();
    for (int i = threadIdx.x; i < N * CY; i += NT) {
        const int sl = i / CY, c = i % CY;
        T[sl * W3 + CY + c] = cmul_is(T[sl * W3 + c], signed_k_mult<N>(slot_freq<N>(sl)));
    }
    __syncthreads();
    fft_lines<N, +1, W3, W3, 1, NT>(T, twN);
    for (int i = threadIdx.x; i < N * CY; i += NT) {
        const int y = i / CY, c = i % CY;
        if (c < cw) {
            const size_t o = base + (size_t)y * H + c;
            ZS[o] = T[y * W3 + c];
            ZGy[o] = T[y * W3 + CY + c];
            ZGz[o] = T[y * W3 + 2 * CY + c];
        }
    }
}

// x inverse: RBX rows (q = z N + y): (E, Fx) from S'', (Fy, Fz) from Gy'', Gz''
template <int N>
__global__ void __launch_bounds__(Pencil<N>::NT) xinv_kernel(const float2 *__restrict__ ZS,
                                                             const float2 *__restrict__ ZGy,
                                                             const float2 *__restrict__ ZGz, FieldPtrs out) {
    constexpr int H = Pencil<N>::H, RBX = Pencil<N>::RBX, NT = Pencil<N>::NT, PW = Pencil<N>::PW,
                  TP = Pencil<N>::TP;
    extern __shared__ __align__(16) float2 sm[];
    float2 *plane = sm;                    // [RBX][PW]
    float2 *Tb = plane + RBX * PW;         // [RBX][TP]
    float2 *twN = Tb + RBX * TP;
    const size_t q0 = (size_t)blockIdx.x * RBX;
    const int r = blockIdx.y;
    const size_t in = ((size_t)r * N * N + q0) * H;
    for (int i = threadIdx.x; i < RBX * H; i += NT) {
        const int row = i / H, c = i % H;
        cp_async8(plane + row * PW + c, ZS + in + i);
        cp_async8(plane + row * PW + H + c, ZGy + in + i);
        cp_async8(plane + row * PW + 2 * H + c, ZGz + in + i);
    }
    load_tw<N>(twN);
    cp_async_wait_all();
    __syncthreads();
    const size_t fo = (size_t)r * out.rot_stride + q0 * N;
    x_pass<N, 0, PW, RBX, TP, NT, RBX>(plane, plane, 0, H, Tb, twN, out.E + fo, out.Fx + fo);
    x_pass<N, 1, PW, RBX, TP, NT, RBX>(plane, plane, 2 * H, H, Tb, twN, out.Fy + fo, out.Fz + fo);
}

// ------------------------------------------- spectral-mode table of a part
// rho2 (N^3) at the centre of an os N grid of zeros (same spacing): original
// node n sits at padded node n + (os - 1) N / 2
template <int N>
__global__ void pad_center_kernel(const float *__restrict__ g, float *__restrict__ out, int np) {
    const int off = (np - N) / 2;
    const size_t total = (size_t)np * np * np;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % np) - off, y = (int)((i / np) % np) - off, z = (int)(i / ((size_t)np * np)) - off;
        const bool in = x >= 0 && x < N && y >= 0 && y < N && z >= 0 && z < N;
        out[i] = in ? __ldg(g + ((size_t)z * N + y) * N + x) : 0.f;
    }
}

// full centred table [kz][ky][kx] (natural order) from the NP half spectrum
// in slot order [kz*][ky*][kx*]: negative kx by Hermitian symmetry, and the
// phase moved to the physical origin by (-1)^(kx+ky+kz)
template <int NP>
__global__ void spectral_complete_kernel(const float2 *__restrict__ spec, float2 *__restrict__ table) {
    constexpr int HP = NP / 2 + 1;
    const size_t total = (size_t)NP * NP * NP;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int kx = (int)(i % NP), ky = (int)((i / NP) % NP), kz = (int)(i / ((size_t)NP * NP));
        float2 v;
        if (2 * kx <= NP) {
            v = __ldg(spec + ((size_t)perm_slot<NP>(kz) * NP + perm_slot<NP>(ky)) * HP + xslot<NP>(kx));
        } else {
            const int mz = (NP - kz) % NP, my = (NP - ky) % NP;
            v = cconj(__ldg(spec + ((size_t)perm_slot<NP>(mz) * NP + perm_slot<NP>(my)) * HP + xslot<NP>(NP - kx)));
        }
        table[i] = ((kx + ky + kz) & 1) ? make_float2(-v.x, -v.y) : v;
    }
}

// -------------------------------------------- natural-order spectrum copy
// spec[kz*][ky*][kx*] (slot order, as left by pass B mode 1) -> out[kz][ky][kx]
template <int N>
__global__ void unpermute_spectrum_kernel(const float2 *__restrict__ spec, float2 *__restrict__ out) {
    constexpr int H = N / 2 + 1;
    const size_t total = (size_t)N * N * H;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int kx = (int)(i % H), ky = (int)((i / H) % N), kz = (int)(i / ((size_t)H * N));
        out[i] = spec[((size_t)perm_slot<N>(kz) * N + perm_slot<N>(ky)) * H + xslot<N>(kx)];
    }
}

// ------------------------------------------------------------- launchers
template <int N>
static cudaError_t set_pencil_attrs() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(xfwd_kernel<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Pencil<N>::smem_xfwd))) return e;
    if ((e = cudaFuncSetAttribute(xfwd_kernel<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Pencil<N>::smem_xfwd))) return e;
    if ((e = cudaFuncSetAttribute(yfwd_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Pencil<N>::smem_yfwd))) return e;
    if ((e = cudaFuncSetAttribute(yinv_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Pencil<N>::smem_yinv))) return e;
    if ((e = cudaFuncSetAttribute(xinv_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Pencil<N>::smem_xinv))) return e;
    if ((e = cudaFuncSetAttribute(passB_kernel<N, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PassB<N>::smem))) return e;
    if ((e = cudaFuncSetAttribute(passB_kernel<N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PassB<N>::smem))) return e;
    if ((e = cudaFuncSetAttribute(passB_kernel<N, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PassB<N>::smem))) return e;
    return cudaSuccess;
}

template <int N>
static cudaError_t set_smem_attrs() {
    cudaError_t e;
    if ((e = set_pencil_attrs<N>())) return e;
    if ((e = cudaFuncSetAttribute(passA_kernel<N, SRC_RAW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PassA<N>::smem))) return e;
    if ((e = cudaFuncSetAttribute(passA_kernel<N, SRC_PLANES>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PassA<N>::smem))) return e;
    if ((e = cudaFuncSetAttribute(passA_kernel<N, SRC_TEX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PassA<N>::smem))) return e;
    // two CTAs per SM (136 KB of shared memory) leave the rest of the unified
    // L1 to the texture cache that the fused resample reads through
    if ((e = cudaFuncSetAttribute(passA_kernel<N, SRC_TEX>, cudaFuncAttributePreferredSharedMemoryCarveout, 62))) return e;
    if ((e = cudaFuncSetAttribute(passB_kernel<N, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PassB<N>::smem))) return e;
    if ((e = cudaFuncSetAttribute(passB_kernel<N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PassB<N>::smem))) return e;
    if ((e = cudaFuncSetAttribute(passB_kernel<N, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PassB<N>::smem))) return e;
    if ((e = cudaFuncSetAttribute(passC_kernel<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PassC<N>::smem))) return e;
    if constexpr (N >= 64 && N <= 128) {  // the autotuner's tile candidates
        if ((e = cudaFuncSetAttribute(passB_kernel<N, 0, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PassB<N, 16>::smem))) return e;
        if ((e = cudaFuncSetAttribute(passC_kernel<N, false, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PassC<N, 16>::smem))) return e;
        if ((e = cudaFuncSetAttribute(passC_kernel<N, false, 0, (N == 128 ? 256 : 0), 1, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)passC_bulk_smem<N, 0, (N == 128 ? 256 : 0)>()))) return e;
        if constexpr (N == 128) {
            if ((e = cudaFuncSetAttribute(passC_kernel<N, false, 0, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PassC<N, 0, 256>::smem))) return e;
            if ((e = cudaFuncSetAttribute(passC_kernel<N, false, 0, 256, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PassC<N, 0, 256>::smem))) return e;
            if ((e = cudaFuncSetAttribute(passC_kernel<N, false, 0, 256, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PassC<N, 0, 256>::smem))) return e;
            if ((e = cudaFuncSetAttribute(passC_kernel<N, false, 0, 0, 1, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)passC_bulk_smem<N>()))) return e;
            if ((e = cudaFuncSetAttribute(passC_kernel<N, false, 0, 256, 1, false, true, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)passC_bulk_smem<N, 0, 256>()))) return e;
        }
    }
    if ((e = cudaFuncSetAttribute(passC_kernel<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PassC<N>::smem))) return e;
    if ((e = cudaFuncSetAttribute(passB_torque_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(sizeof(float2) * (3 * (size_t)N * PassB<N>::CW + N)))))
        return e;
    return cudaSuccess;
}

template <int N, int SRC>
static cudaError_t launch_passA(const float *rho, const float *rot9, float2 *X1, int nrot, cudaStream_t st,
                               cudaTextureObject_t tex = 0, const int *box = nullptr) {
    passA_kernel<N, SRC><<<dim3(N, nrot), PassA<N>::NT, PassA<N>::smem, st>>>(rho, rot9, X1, tex, box);
    return cudaGetLastError();
}
template <int N>
static cudaError_t launch_pad_slices(const float *g, float *slab, size_t pitch_floats, cudaStream_t st) {
    pad_slices_kernel<N><<<4 * 148, 256, 0, st>>>(g, slab, pitch_floats);
    return cudaGetLastError();
}
template <int N>
static cudaError_t launch_support(const float *g, unsigned *masks, int *box, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(masks, 0, kSupportMaskWords * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    support_masks_kernel<N><<<N, N, 0, st>>>(g, masks);
    support_box_kernel<N><<<1, 32, 0, st>>>(masks, box);
    return cudaGetLastError();
}
template <int N>
static cudaError_t launch_resample_chunk(const float *rho, const float *rot9, float *out, int nrot, cudaStream_t st) {
    resample_chunk_kernel<N><<<dim3((N / kRsX) * (N / kRsY) * (N / kRsZ), nrot), kRsX * kRsY, 0, st>>>(rho, rot9, out);
    return cudaGetLastError();
}
template <int N, int CWO = 0>
static cudaError_t launch_passB(const float2 *X1, const float2 *R1hat, float2 *Y1, float2 *Y2, int nrot,
                                cudaStream_t st) {
    using PB = PassB<N, CWO>;
    passB_kernel<N, 0, CWO><<<dim3(N * PB::H / PB::CW, nrot), PB::NT, PB::smem, st>>>(
        X1, R1hat, Y1, Y2, 0.f, SpecSrc{nullptr, 0, 0}, nullptr);
    return cudaGetLastError();
}
template <int N>
static cudaError_t launch_passB_fwd(const float2 *X1, float2 *spec, float scale, cudaStream_t st) {
    passB_kernel<N, 1><<<dim3(N * PassB<N>::H / PassB<N>::CW, 1), PassB<N>::NT, PassB<N>::smem, st>>>(
        X1, nullptr, spec, nullptr, scale, SpecSrc{nullptr, 0, 0}, nullptr);
    return cudaGetLastError();
}
template <int N>
static cudaError_t launch_passB_spectral(const float2 *table, cudaTextureObject_t tex, int os, const float *rot9,
                                         const float2 *R1hat, float2 *Y1, float2 *Y2, int nrot, cudaStream_t st) {
    constexpr int tiles = (N / 2 + PassB<N>::CW - 1) / PassB<N>::CW;
    passB_kernel<N, 2><<<dim3(N * tiles, nrot), PassB<N>::NT, PassB<N>::smem, st>>>(
        nullptr, R1hat, Y1, Y2, 0.f, SpecSrc{table, os * N, os, tex, table_tex_sc(os * N)}, rot9);
    return cudaGetLastError();
}
template <int N, int RBO = 0, int NTO = 0, int YU = 1, bool PF = false, bool BK = false, int XR1 = 0>
static cudaError_t launch_passC(const float2 *Y1, const float2 *Y2, FieldPtrs out, int nrot, cudaStream_t st) {
    using PC = PassC<N, RBO, NTO>;
    if constexpr (BK) {
        // the bulk copies read whole planes: 16-byte aligned sources
        if (((uintptr_t)Y1 | (uintptr_t)Y2) % 16) return cudaErrorMisalignedAddress;
    }
    passC_kernel<N, false, RBO, NTO, YU, PF, BK, XR1>
        <<<dim3(N, nrot), PC::NT, BK ? passC_bulk_smem<N, RBO, NTO>() : PC::smem, st>>>(Y1, Y2, out, nullptr, 0);
    return cudaGetLastError();
}
template <int N>
static cudaError_t launch_passC_torque(const float2 *Y1, const float2 *Y2, const float2 *YT, size_t yt_stride,
                                       FieldPtrs out, int nrot, cudaStream_t st) {
    passC_kernel<N, true><<<dim3(N, nrot), PassC<N>::NT, PassC<N>::smem, st>>>(Y1, Y2, out, YT, yt_stride);
    return cudaGetLastError();
}
template <int N>
static cudaError_t launch_passB_torque(const float2 *X1, const float2 *Gm, float2 *YT, size_t yt_stride, int nrot,
                                       cudaStream_t st) {
    const size_t sm = sizeof(float2) * (3 * (size_t)N * PassB<N>::CW + N);
    passB_torque_kernel<N><<<dim3(N * PassB<N>::H / PassB<N>::CW, nrot), PassB<N>::NT, sm, st>>>(X1, Gm, YT, yt_stride);
    return cudaGetLastError();
}
template <int N>
static cudaError_t launch_moment_fields(const float *Fx, const float *Fy, const float *Fz, float *G, cudaStream_t st) {
    moment_fields_kernel<N><<<4 * 148, 256, 0, st>>>(Fx, Fy, Fz, G);
    return cudaGetLastError();
}
template <int N>
static cudaError_t launch_xfwd(const float *planes, float2 *Xa, int nrot, cudaStream_t st) {
    xfwd_kernel<N, false><<<dim3(N * N / Pencil<N>::RBX, nrot), Pencil<N>::NT, Pencil<N>::smem_xfwd, st>>>(
        planes, Xa, 0, nullptr, nullptr);
    return cudaGetLastError();
}
template <int N>
static cudaError_t launch_xfwd_tex(cudaTextureObject_t tex, const int *box, const float *rot9, float2 *Xa, int nrot,
                                   cudaStream_t st) {
    xfwd_kernel<N, true><<<dim3(N * N / Pencil<N>::RBX, nrot), Pencil<N>::NT, Pencil<N>::smem_xfwd, st>>>(
        nullptr, Xa, tex, rot9, box);
    return cudaGetLastError();
}
template <int N>
static cudaError_t launch_yfwd(const float2 *Xa, float2 *X1, int nrot, cudaStream_t st) {
    yfwd_kernel<N><<<dim3(N * Pencil<N>::NCY, nrot), Pencil<N>::NT, Pencil<N>::smem_yfwd, st>>>(Xa, X1);
    return cudaGetLastError();
}
template <int N>
static cudaError_t launch_yinv(const float2 *Y1, const float2 *Y2, float2 *ZS, float2 *ZGy, float2 *ZGz, int nrot,
                               cudaStream_t st) {
    yinv_kernel<N><<<dim3(N * Pencil<N>::NCY, nrot), Pencil<N>::NT, Pencil<N>::smem_yinv, st>>>(Y1, Y2, ZS, ZGy, ZGz);
    return cudaGetLastError();
}
template <int N>
static cudaError_t launch_xinv(const float2 *ZS, const float2 *ZGy, const float2 *ZGz, FieldPtrs out, int nrot,
                               cudaStream_t st) {
    xinv_kernel<N><<<dim3(N * N / Pencil<N>::RBX, nrot), Pencil<N>::NT, Pencil<N>::smem_xinv, st>>>(ZS, ZGy, ZGz, out);
    return cudaGetLastError();
}
template <int N>
static cudaError_t launch_pad_center(const float *g, float *out, int np, cudaStream_t st) {
    pad_center_kernel<N><<<4 * 148, 256, 0, st>>>(g, out, np);
    return cudaGetLastError();
}
template <int NP>
static cudaError_t launch_spectral_complete(const float2 *spec, float2 *table, cudaStream_t st) {
    spectral_complete_kernel<NP><<<8 * 148, 256, 0, st>>>(spec, table);
    return cudaGetLastError();
}
template <int N>
static cudaError_t launch_unpermute(const float2 *spec, float2 *out, cudaStream_t st) {
    unpermute_spectrum_kernel<N><<<148, 256, 0, st>>>(spec, out);
    return cudaGetLastError();
}

// ------------------------------------------------- one-launch field build
// A whole batch of pairs in one launch over a device work queue: each block
// takes the next item by ticket (a global counter) and runs it with the same
// bodies as the per-pass kernels (256 threads: pass C at 128^3 with 256
// instead of 512); an item is one block's worth of pass A, B or C of one
// (pair, rotation chunk).  The launch has one block per item and no block
// loops: a looping block lets the compiler hoist the bodies' per-thread
// terms out of the loop, and with every body in one function that spilled
// 2.1 KB per thread at the 128-register cap; the hardware block scheduler
// keeps the SMs fed instead.  Tickets go out in the order blocks start, and
// an item waits only for items with smaller tickets (its pass's producers,
// or the previous user of its intermediates or outputs), so every wait is
// for a block that has already started.  Waits are bounded: after
// spin_limit polls the block sets the status word to PERSIST_TIMEOUT, and
// every block that starts later returns at once.
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed_s32(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t kPersistSmem =
    cmax(cmax(cmax(PassA<64>::smem, PassA<96>::smem), cmax(PassA<128>::smem, PassB<64>::smem)),
         cmax(cmax(PassB<96>::smem, PassB<128>::smem),
              cmax(passC_bulk_smem<64>(), cmax(passC_bulk_smem<96>(), passC_bulk_smem<128>()))));

template <int N>
__device__ __forceinline__ void persist_item(const PersistSeg &g, int local) {
    static_assert(PassA<N>::NT == kPersistNT && PassB<N>::NT == kPersistNT, "256-thread passes A and B");
    constexpr int BT = N * PassB<N>::H / PassB<N>::CW;  // pass B column tiles per rotation
    if (g.pass == 0) {
        passA_body<N, SRC_TEX>(nullptr, g.rot9, g.X1, g.tex, g.box, local % N, local / N);
    } else if (g.pass == 1) {
        passB_body<N, 0, true>(g.X1, g.R1hat, g.Y1, g.Y2, 0.f, SpecSrc{nullptr, 0, 0}, nullptr, local % BT,
                               local / BT);
    } else {
        passC_body<N, false, kPersistNT, true, 0, 1, false, true>(g.Y1, g.Y2, g.out, nullptr, 0, local % N,
                                                                 local / N);
    }
}

__global__ void __launch_bounds__(kPersistNT, 2)
    queue_kernel(const PersistSeg *__restrict__ segs, const int *__restrict__ lut, int nseg, int total,
                 unsigned *queue, unsigned *counters, int *status, long long spin_limit) {
    __shared__ int s_item, s_seg, s_stop;
    if (threadIdx.x == 0) {
        const int it = (int)atomicAdd(queue, 1u);
        int stop = it >= total || ld_relaxed_s32(status) != PERSIST_OK;
        int sg = 0;
        if (!stop) {
            // the run holding item it: from the run holding item it & ~255, forward
            sg = __ldg(lut + (it >> 8));
            while (sg + 1 < nseg && __ldg(&segs[sg + 1].base) <= it) ++sg;
            for (int d = 0; d < 2 && !stop; ++d) {
                const int c = segs[sg].dep[d];
                if (c < 0) continue;
                const unsigned target = (unsigned)segs[sg].dep_target[d];
                long long k = 0;
                while (ld_acquire_u32(counters + c) < target) {
                    if (++k > spin_limit || ld_relaxed_s32(status) != PERSIST_OK) {
                        atomicCAS(status, PERSIST_OK, PERSIST_TIMEOUT);
                        stop = 1;
                        break;
                    }
                    __nanosleep(256);
                }
            }
            // pass C items read their producers' output by bulk copies (the
            // async proxy) that this thread issues: order them after the
            // generic-proxy writes it has just acquired
            asm volatile("fence.proxy.async.global;" ::: "memory");
        }
        s_item = it;
        s_seg = sg;
        s_stop = stop;
    }
    __syncthreads();
    if (s_stop) return;
    const PersistSeg &g = segs[s_seg];
    const int local = s_item - g.base + g.first;
    if (g.n == 64) persist_item<64>(g, local);
    else if (g.n == 96) persist_item<96>(g, local);
    else persist_item<128>(g, local);
    __syncthreads();  // every thread's writes of the item are done
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(counters + g.done, 1u);
    }
}

cudaError_t persist_init() {
    cudaError_t e = cudaFuncSetAttribute(queue_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPersistSmem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(queue_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
}
size_t persist_smem() { return kPersistSmem; }
int persist_blocks_per_sm() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, queue_kernel, kPersistNT, kPersistSmem) != cudaSuccess)
        return 0;
    return nb;
}
cudaError_t run_persistent(const PersistSeg *d_segs, const int *d_lut, int nseg, int total, unsigned *d_queue,
                           unsigned *d_counters, int *d_status, long long spin_limit, cudaStream_t st) {
    queue_kernel<<<total, kPersistNT, kPersistSmem, st>>>(d_segs, d_lut, nseg, total, d_queue, d_counters, d_status,
                                                           spin_limit);
    return cudaGetLastError();
}

#define HF_DISPATCH(n, call)                                \
    switch (n) {                                            \
        case 32: { constexpr int NN = 32; return call; }    \
        case 64: { constexpr int NN = 64; return call; }    \
        case 96: { constexpr int NN = 96; return call; }    \
        case 128: { constexpr int NN = 128; return call; }  \
        default: return cudaErrorInvalidValue;              \
    }
// kernels built for every size, the pencil pipeline's 256 included
#define HF_DISPATCH_ALL(n, call)                            \
    switch (n) {                                            \
        case 32: { constexpr int NN = 32; return call; }    \
        case 64: { constexpr int NN = 64; return call; }    \
        case 96: { constexpr int NN = 96; return call; }    \
        case 128: { constexpr int NN = 128; return call; }  \
        case 256: { constexpr int NN = 256; return call; }  \
        default: return cudaErrorInvalidValue;              \
    }

cudaError_t fft_init_attrs(int n) {
    if (n == 256) return set_pencil_attrs<256>();
    HF_DISPATCH(n, set_smem_attrs<NN>());
}
cudaError_t run_xfwd(int n, const float *planes, float2 *Xa, int nrot, cudaStream_t st) {
    HF_DISPATCH_ALL(n, launch_xfwd<NN>(planes, Xa, nrot, st));
}
cudaError_t run_xfwd_tex(int n, cudaTextureObject_t tex, const int *box, const float *rot9, float2 *Xa, int nrot,
                         cudaStream_t st) {
    HF_DISPATCH_ALL(n, launch_xfwd_tex<NN>(tex, box, rot9, Xa, nrot, st));
}
cudaError_t run_yfwd(int n, const float2 *Xa, float2 *X1, int nrot, cudaStream_t st) {
    HF_DISPATCH_ALL(n, launch_yfwd<NN>(Xa, X1, nrot, st));
}
cudaError_t run_yinv(int n, const float2 *Y1, const float2 *Y2, float2 *ZS, float2 *ZGy, float2 *ZGz, int nrot,
                     cudaStream_t st) {
    HF_DISPATCH_ALL(n, launch_yinv<NN>(Y1, Y2, ZS, ZGy, ZGz, nrot, st));
}
cudaError_t run_xinv(int n, const float2 *ZS, const float2 *ZGy, const float2 *ZGz, FieldPtrs out, int nrot,
                     cudaStream_t st) {
    HF_DISPATCH_ALL(n, launch_xinv<NN>(ZS, ZGy, ZGz, out, nrot, st));
}
cudaError_t run_passA(int n, const float *rho, const float *rot9, float2 *X1, int nrot, cudaStream_t st) {
    HF_DISPATCH(n, (launch_passA<NN, SRC_RAW>(rho, rot9, X1, nrot, st)));
}
cudaError_t run_passA_tex(int n, cudaTextureObject_t tex, const int *box, const float *rot9, float2 *X1, int nrot,
                          cudaStream_t st) {
    HF_DISPATCH(n, (launch_passA<NN, SRC_TEX>(nullptr, rot9, X1, nrot, st, tex, box)));
}
cudaError_t run_passA_planes(int n, const float *planes, float2 *X1, int nrot, cudaStream_t st) {
    HF_DISPATCH(n, (launch_passA<NN, SRC_PLANES>(planes, nullptr, X1, nrot, st)));
}
cudaError_t run_resample_chunk(int n, const float *rho, const float *rot9, float *out, int nrot, cudaStream_t st) {
    HF_DISPATCH_ALL(n, launch_resample_chunk<NN>(rho, rot9, out, nrot, st));
}
cudaError_t run_support(int n, const float *g, unsigned *masks, int *box, cudaStream_t st) {
    HF_DISPATCH_ALL(n, launch_support<NN>(g, masks, box, st));
}
cudaError_t run_pad_slices(int n, const float *g, float *slab, size_t pitch_floats, cudaStream_t st) {
    HF_DISPATCH_ALL(n, launch_pad_slices<NN>(g, slab, pitch_floats, st));
}
cudaError_t run_passB(int n, const float2 *X1, const float2 *R1hat, float2 *Y1, float2 *Y2, int nrot, cudaStream_t st,
                      int tile) {
    if (tile == 1) {  // 16 columns per CTA
        switch (n) {
            case 64: return launch_passB<64, 16>(X1, R1hat, Y1, Y2, nrot, st);
            case 96: return launch_passB<96, 16>(X1, R1hat, Y1, Y2, nrot, st);
            case 128: return launch_passB<128, 16>(X1, R1hat, Y1, Y2, nrot, st);
            default: break;
        }
    }
    HF_DISPATCH_ALL(n, launch_passB<NN>(X1, R1hat, Y1, Y2, nrot, st));
}
cudaError_t run_passB_forward(int n, const float2 *X1, float2 *spec, float scale, cudaStream_t st) {
    HF_DISPATCH_ALL(n, launch_passB_fwd<NN>(X1, spec, scale, st));
}
cudaError_t run_passC(int n, const float2 *Y1, const float2 *Y2, FieldPtrs out, int nrot, cudaStream_t st, int tile) {
    if (tile == 1) {  // 16 rows per x batch
        switch (n) {
            case 64: return launch_passC<64, 16>(Y1, Y2, out, nrot, st);
            case 96: return launch_passC<96, 16>(Y1, Y2, out, nrot, st);
            case 128: return launch_passC<128, 16>(Y1, Y2, out, nrot, st);
            default: break;
        }
    } else if (tile == 2 && n == 128) {  // 256 threads per CTA
        return launch_passC<128, 0, 256>(Y1, Y2, out, nrot, st);
    } else if (tile == 3 && n == 128) {  // and an L2 prefetch of the Gz' plane
        return launch_passC<128, 0, 256, 1, true>(Y1, Y2, out, nrot, st);
    } else if (tile == 4 && n == 128) {  // and two y-stage items' loads in flight
        return launch_passC<128, 0, 256, 2, true>(Y1, Y2, out, nrot, st);
    } else if (tile == 5) {  // planes staged by bulk copies (256 threads at 128^3)
        switch (n) {
            case 64: return launch_passC<64, 0, 0, 1, false, true>(Y1, Y2, out, nrot, st);
            case 96: return launch_passC<96, 0, 0, 1, false, true>(Y1, Y2, out, nrot, st);
            case 128: return launch_passC<128, 0, 256, 1, false, true>(Y1, Y2, out, nrot, st);
            default: break;
        }
    } else if (tile == 6 && n == 128) {  // planes staged by bulk copies, 512 threads per CTA
        return launch_passC<128, 0, 0, 1, false, true>(Y1, Y2, out, nrot, st);
    } else if (tile == 7 && n == 128) {  // as tile 5, the x inverse with radix 16 x 8 (16-point stage 1)
        return launch_passC<128, 0, 256, 1, false, true, 16>(Y1, Y2, out, nrot, st);
    }
    HF_DISPATCH(n, launch_passC<NN>(Y1, Y2, out, nrot, st));
}
cudaError_t run_pad_center(int n, const float *g, float *out, int np, cudaStream_t st) {
    HF_DISPATCH_ALL(n, launch_pad_center<NN>(g, out, np, st));
}
cudaError_t run_spectral_complete(int np, const float2 *spec, float2 *table, cudaStream_t st) {
    HF_DISPATCH_ALL(np, launch_spectral_complete<NN>(spec, table, st));
}
cudaError_t run_passB_spectral(int n, const float2 *table, cudaTextureObject_t tex, int os, const float *rot9,
                               const float2 *R1hat, float2 *Y1, float2 *Y2, int nrot, cudaStream_t st) {
    HF_DISPATCH_ALL(n, launch_passB_spectral<NN>(table, tex, os, rot9, R1hat, Y1, Y2, nrot, st));
}
// the table as stacked, wrap-padded (np+1)^2 slices, sc to a texture row:
// texel (X, Y) of the width x height slab is cell (X mod (np+1), Y mod (np+1))
// of slice (Y / (np+1)) sc + X / (np+1), indices np wrapping to 0
__global__ void pad_table_kernel(const float2 *__restrict__ table, int np, int sc, float2 *__restrict__ slab,
                                 int width, int height) {
    const size_t total = (size_t)width * height;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int X = (int)(i % width), Y = (int)(i / width);
        const int z = (Y / (np + 1)) * sc + X / (np + 1);
        const int lx = X % (np + 1), ly = Y % (np + 1);
        slab[i] = z < np ? table[((size_t)z * np + (ly == np ? 0 : ly)) * np + (lx == np ? 0 : lx)]
                         : make_float2(0.f, 0.f);
    }
}
void table_tex_layout(int np, int *width, int *height) {
    const int sc = table_tex_sc(np);
    *width = sc * (np + 1);
    *height = ((np + sc - 1) / sc) * (np + 1);
}
cudaError_t run_pad_table(const float2 *table, int np, float2 *slab, cudaStream_t st) {
    int w = 0, h = 0;
    table_tex_layout(np, &w, &h);
    pad_table_kernel<<<8 * 148, 256, 0, st>>>(table, np, table_tex_sc(np), slab, w, h);
    return cudaGetLastError();
}
cudaError_t run_passB_torque(int n, const float2 *X1, const float2 *Gm, float2 *YT, size_t yt_stride, int nrot,
                             cudaStream_t st) {
    HF_DISPATCH(n, launch_passB_torque<NN>(X1, Gm, YT, yt_stride, nrot, st));
}
cudaError_t run_passC_torque(int n, const float2 *Y1, const float2 *Y2, const float2 *YT, size_t yt_stride,
                             FieldPtrs out, int nrot, cudaStream_t st) {
    HF_DISPATCH(n, launch_passC_torque<NN>(Y1, Y2, YT, yt_stride, out, nrot, st));
}
cudaError_t run_moment_fields(int n, const float *Fx, const float *Fy, const float *Fz, float *G, cudaStream_t st) {
    HF_DISPATCH_ALL(n, launch_moment_fields<NN>(Fx, Fy, Fz, G, st));
}
cudaError_t run_unpermute(int n, const float2 *spec, float2 *out, cudaStream_t st) {
    HF_DISPATCH_ALL(n, launch_unpermute<NN>(spec, out, st));
}

// ------------------------------------------------- bulk-copy wait checks
// The bulk-staged kernels count a wait for their copies that gave up in
// g_bulk_timeouts.  The self test runs the same copy and bounded wait in one
// block on a 4 KB buffer: plain, the buffer comes back unchanged; planted,
// the mbarrier expects 16 bytes more than the copy brings, so the wait runs
// out (twice its bound) and counts itself, with the copy itself complete.
int bulk_timeouts(bool reset) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_bulk_timeouts, sizeof v) != cudaSuccess) return -1;
    if (reset) {
        const int z = 0;
        if (cudaMemcpyToSymbol(g_bulk_timeouts, &z, sizeof z) != cudaSuccess) return -1;
    }
    return v;
}

constexpr int kSelfTestBytes = 4096;

__global__ void bulk_selftest_kernel(const float4 *__restrict__ src, float4 *__restrict__ dst, int plant) {
    __shared__ __align__(16) float4 buf[kSelfTestBytes / 16];
    __shared__ __align__(8) unsigned long long mbar;
    if (threadIdx.x == 0) {
        mbar_init1(&mbar);
        mbar_expect(&mbar, kSelfTestBytes + (plant ? 16u : 0u));
        fence_proxy_async_smem();
        bulk_g2s(buf, src, kSelfTestBytes, &mbar);
    }
    __syncthreads();
    mbar_wait_bounded(&mbar, 0);
    for (int i = threadIdx.x; i < kSelfTestBytes / 16; i += blockDim.x) dst[i] = buf[i];
}

cudaError_t run_bulk_selftest(const void *src, void *dst, int plant, cudaStream_t st) {
    if (((uintptr_t)src | (uintptr_t)dst) % 16) return cudaErrorMisalignedAddress;
    bulk_selftest_kernel<<<1, 128, 0, st>>>(reinterpret_cast<const float4 *>(src), reinterpret_cast<float4 *>(dst),
                                           plant);
    return cudaGetLastError();
}
int bulk_selftest_bytes() { return kSelfTestBytes; }

// Never launched: its address names this file's device-code module, which
// hf_ctx_preload loads whole.
__global__ void module_anchor_fft_kernel() {}
const void *module_anchor_fft() { return (const void *)&module_anchor_fft_kernel; }

}  // namespace hf
