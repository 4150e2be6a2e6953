// hf_tc.cu -- the y stages of the 256^3 pencil pipeline on the tensor cores
// (precision variant): every length-256 complex DFT along y (Eq. 7a forward,
// Eq. 7b inverse) runs as two small DFT-matrix GEMMs, 256 = 16 x 16:
//
//   forward, y = 16 n1 + n2, ky = k1 + 16 k2:
//     stage 1   Y[k1][n2]  = sum_n1 W16^(n1 k1) x[16 n1 + n2]      (GEMM)
//     twiddle   Y[k1][n2] *= W256^(n2 k1)                          (FP32)
//     stage 2   X[k1 + 16 k2] = sum_n2 W16^(n2 k2) Y[k1][n2]       (GEMM)
//   inverse, ky = k1 + 16 k2, y = n2 + 16 n1: the same with the roles of
//     the digits exchanged and conjugate matrices.
//
// A CTA owns CT = 32 grid columns (flattened (z, kx) of one rotation), so a
// stage is one real GEMM D[512 x 32] = A[512 x 32] B[32 x 32]: rows of A are
// (group digit, column), its K the (other digit, re/im) pairs, B the 16-point
// DFT in real 2x2-block form.  Operands are split into hi + lo parts in BF16
// or FP16 (v = hi + lo exactly up to the lo rounding); each K step issues
// hi*hi + hi*lo + lo*hi (the lo*lo term, ~2^-16 relative for BF16, dropped)
// with FP32 accumulation in tensor memory (tcgen05.mma kind::f16, M = 128,
// N = 32, K = 16, both operands K-major without swizzle).  FP16 operands are
// scaled per tile by a power of two into range, and their lo parts by 2^11
// into a second accumulator, so that no lo part is subnormal.  The twiddles,
// the Gy multiplier and the rescaling run in FP32 in the epilogues.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "hf_dft.cuh"
#include "hf_internal.h"

namespace hf {
namespace tc {

constexpr int N = 256, H = N / 2 + 1, RD = 16;  // N = RD * RD
constexpr int CT = 32;                          // grid columns per CTA
constexpr int M = CT * RD;                      // 512 GEMM rows per stage
constexpr int MT = M / 128;                     // 4 M tiles of 128 rows
constexpr int KR = 2 * RD;                      // 32 real K per stage
constexpr int NR = 2 * RD;                      // 32 real outputs per row
constexpr int NT = 256;
constexpr uint32_t A_BYTES = (uint32_t)M * KR * 2;   // 32 KB per part
constexpr uint32_t B_BYTES = (uint32_t)NR * KR * 2;  // 2 KB per part
constexpr size_t SMEM = 2 * (size_t)A_BYTES + 2 * (size_t)B_BYTES + 128;
// FP32 accumulator columns: one 32-column D per M tile; FP16 keeps the lo
// products in a second set (see split2)
template <bool F16>
__host__ __device__ constexpr uint32_t tmem_cols() {
    return (F16 ? 2u : 1u) * MT * NR;
}
// FP16 lo parts are stored times 2^11: a lo below FP16's normal range would
// be flushed in the products, costing 2^-11 of every value under 1/8 of the
// tile's largest
constexpr float LO_UP = 2048.f, LO_DOWN = 1.f / 2048.f;
constexpr unsigned long long WAIT_NS = 200ull * 1000 * 1000;  // bound on one wait for an MMA group
static_assert(N * H % CT == 0, "columns of a rotation split into whole CTAs");

// cos / sin (2 pi t / 256), t < 256, rounded once from double
struct Trig256 {
    float c[N], s[N];
};
constexpr Trig256 make_trig() {
    Trig256 t{};
    for (int j = 0; j < N; ++j) {
        t.c[j] = (float)ct::trig(j, N, 0);
        t.s[j] = (float)ct::trig(j, N, 1);
    }
    return t;
}
__device__ const Trig256 g_trig = make_trig();
__device__ int g_tc_timeouts = 0;

// byte offset of element (row, k) of a K-major operand with 32 K-values per
// row: 8 x 16-byte core matrices, K-adjacent ones 128 B apart (LBO), 8-row
// groups 512 B apart (SBO)
__device__ __forceinline__ uint32_t kmaj_off(int row, int k) {
    return (uint32_t)((row >> 3) * 512 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start >> 4, LBO = 128 B, SBO = 512 B,
// descriptor version 1 (bit 46), base offset 0, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(512 >> 4) << 32) |
           (1ull << 46);
}
// instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9, 10-12 = 1) or FP16 (0), both K-major, N >> 3 at bit 17,
// M >> 4 at bit 24
template <bool F16>
__host__ __device__ constexpr uint32_t idesc() {
    return (1u << 4) | ((F16 ? 0u : 1u) << 7) | ((F16 ? 0u : 1u) << 10) | ((uint32_t)(NR >> 3) << 17) |
           ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// bounded wait for the MMA group's commit; false after WAIT_NS
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    const unsigned long long t0 = now_ns();
    while (!mbar_try_wait(mbar, parity))
        if (now_ns() - t0 > WAIT_NS) return false;
    return true;
}

// 16 consecutive FP32 columns of this thread's TMEM lane (warp w reads lanes
// 32 (w % 4) .. + 31); the wait is in the same statement so that no use of
// the registers can be scheduled before the load completes
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 accumulator columns [16 h, 16 h + 16) of M tile t for this thread's
// lane: the hi products plus (FP16) the rescaled lo products
template <bool F16>
__device__ __forceinline__ void load_acc(uint32_t tbase, int sp, int t, int h, float (&v)[16]) {
    const uint32_t a = tbase + ((uint32_t)(32 * sp) << 16) + (uint32_t)(t * NR + 16 * h);
    tmem_ld16(a, v);
    if constexpr (F16) {
        float w[16];
        tmem_ld16(a + MT * NR, w);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = fmaf(w[i], LO_DOWN, v[i]);
    }
}

// (re, im) -> packed hi pair and lo pair
template <bool F16>
__device__ __forceinline__ void split2(float re, float im, uint32_t &hi, uint32_t &lo) {
    if constexpr (F16) {
        const __half hr = __float2half_rn(re), hm = __float2half_rn(im);
        const __half lr = __float2half_rn((re - __half2float(hr)) * LO_UP);
        const __half lm = __float2half_rn((im - __half2float(hm)) * LO_UP);
        const __half2 h2 = __halves2half2(hr, hm), l2 = __halves2half2(lr, lm);
        hi = *reinterpret_cast<const uint32_t *>(&h2);
        lo = *reinterpret_cast<const uint32_t *>(&l2);
    } else {
        const __nv_bfloat16 hr = __float2bfloat16_rn(re), hm = __float2bfloat16_rn(im);
        const __nv_bfloat16 lr = __float2bfloat16_rn(re - __bfloat162float(hr));
        const __nv_bfloat16 lm = __float2bfloat16_rn(im - __bfloat162float(hm));
        const __nv_bfloat162 h2 = __halves2bfloat162(hr, hm), l2 = __halves2bfloat162(lr, lm);
        hi = *reinterpret_cast<const uint32_t *>(&h2);
        lo = *reinterpret_cast<const uint32_t *>(&l2);
    }
}
template <bool F16>
__device__ __forceinline__ void split1(float v, uint16_t &hi, uint16_t &lo) {
    if constexpr (F16) {
        const __half h = __float2half_rn(v), l = __float2half_rn((v - __half2float(h)) * LO_UP);
        hi = __half_as_ushort(h);
        lo = __half_as_ushort(l);
    } else {
        const __nv_bfloat16 h = __float2bfloat16_rn(v), l = __float2bfloat16_rn(v - __bfloat162float(h));
        hi = __bfloat16_as_ushort(h);
        lo = __bfloat16_as_ushort(l);
    }
}

__device__ __forceinline__ float pi_k_signed(int k) {  // pi k~, 0 at the Nyquist index
    return (2 * k == N) ? 0.0f : 3.14159265358979323846f * (float)(k < N / 2 ? k : k - N);
}

// One length-256 y transform per column of a 32-column tile.  Forward
// (INV = false): src rows in natural y order, dst rows in the digit-permuted
// slot order of the FP32 pipeline (slot 16 k1 + k2 for ky = k1 + 16 k2).
// Inverse: src rows in slot order, dst in natural y; blockIdx.z = 0 runs two
// transforms from one load of src0, src0 -> dst0 and src0 times i pi ky~ ->
// dst1, and blockIdx.z = 1 runs src1 -> dst2.
//
// Operand staging: every thread writes its rows' K-values as 16-byte vectors
// (4 complex values of consecutive K digit b), so a warp's stores fill whole
// 128-byte rows of the K-major core matrices without bank conflicts; the
// element locations (kmaj_off) are those the descriptors read.
template <bool INV, bool F16>
__global__ void __launch_bounds__(NT, 2) y_tc_kernel(const float2 *__restrict__ src0, const float2 *__restrict__ src1,
                                                     float2 *__restrict__ dst0, float2 *__restrict__ dst1,
                                                     float2 *__restrict__ dst2) {
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *Ahi = smem, *Alo = smem + A_BYTES;
    uint8_t *Bhi = smem + 2 * A_BYTES, *Blo = Bhi + B_BYTES;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(Blo + B_BYTES);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
    float *red = reinterpret_cast<float *>(tslot + 1) + 1;  // 8 warp maxima (16-byte aligned start not needed)

    // after a timed-out wait anywhere, later blocks leave at once (their
    // outputs are invalid either way) so that a failure ends quickly
    if (*reinterpret_cast<volatile int *>(&g_tc_timeouts) != 0) return;
    const int set = blockIdx.z;
    const float2 *src = set == 1 ? src1 : src0;
    const int ntr = (INV && set == 0) ? 2 : 1;  // transforms of this block
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int f = blockIdx.x * CT + lane;  // flattened (z, kx slot) column of this lane
    const int zc = f / H, cc = f - zc * H;
    const size_t col = (size_t)blockIdx.y * N * N * H + (size_t)zc * N * H + cc;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                     "r"(tmem_cols<F16>())
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 32) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // B: the 16-point DFT W = exp(-+ 2 pi i b j / 16) in real form; row jj =
    // 2 j + (0 re | 1 im) of the output, column kk = 2 b + (0 re | 1 im) of
    // the input: [Wr -Wi; Wi Wr]
    for (int i = threadIdx.x; i < NR * KR; i += NT) {
        const int jj = i / KR, kk = i % KR;
        const int j = jj >> 1, b = kk >> 1;
        const int t = ((b * j) & 15) * (N / RD);
        const float c = g_trig.c[t], s = INV ? g_trig.s[t] : -g_trig.s[t];
        const float v = (jj & 1) == 0 ? ((kk & 1) == 0 ? c : -s) : ((kk & 1) == 0 ? s : c);
        uint16_t h, l;
        split1<F16>(v, h, l);
        *reinterpret_cast<uint16_t *>(Bhi + kmaj_off(jj, kk)) = h;
        *reinterpret_cast<uint16_t *>(Blo + kmaj_off(jj, kk)) = l;
    }
    // stage-1 operand rows: thread (warp w) holds, for 8 (group digit a,
    // K block m) pairs p = w + 8 q, the 4 input rows of K digits b = 4 m ..
    // 4 m + 3 of group a.  Forward: input row y = a + 16 b; inverse: the row
    // of slot order holding frequency a + 16 b, i.e. slot 16 a + b.
    float2 x[32];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int p = warp + 8 * q, a = p >> 2, m = p & 3;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int b = 4 * m + u;
            const int y = INV ? 16 * a + b : a + 16 * b;
            x[4 * q + u] = src[col + (size_t)y * H];
        }
    }
    // the tensor-memory address that warp 0's allocation wrote, and the
    // initialised mbarrier, are visible to every thread after this barrier
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tbase = *tslot;
    const uint32_t sAhi = su32(Ahi), sAlo = su32(Alo), sBhi = su32(Bhi), sBlo = su32(Blo), sbar = su32(mbar);
    constexpr uint32_t ID = idesc<F16>();
    auto issue = [&]() {
#pragma unroll
        for (int t = 0; t < MT; ++t) {
            const uint32_t d = tbase + (uint32_t)(t * NR);
            const uint32_t dl = F16 ? d + MT * NR : d;  // accumulator of the lo products
#pragma unroll
            for (int ks = 0; ks < KR / 16; ++ks) {
                const uint32_t ao = (uint32_t)(t * 128 / 8 * 512 + ks * 256), bo = (uint32_t)(ks * 256);
                mma(d, smem_desc(sAhi + ao), smem_desc(sBhi + bo), ID, ks > 0 ? 1u : 0u);
                mma(dl, smem_desc(sAhi + ao), smem_desc(sBlo + bo), ID, (F16 && ks == 0) ? 0u : 1u);
                mma(dl, smem_desc(sAlo + ao), smem_desc(sBhi + bo), ID, 1u);
            }
        }
        mma_commit(sbar);
    };
    const int sp = warp & 3;
    bool ok = true;
    uint32_t phase = 0;
    for (int tr = 0; tr < ntr && ok; ++tr) {
        float2 *dst = set == 1 ? dst2 : (tr == 0 ? dst0 : dst1);
        if (INV && set == 0 && tr == 1) {  // Gy = i pi ky~ S, ky~ of the row's slot (S is no longer needed)
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const int q = i >> 2, u = i & 3, p = warp + 8 * q;
                x[i] = cmul_is(x[i], pi_k_signed(slot_freq<N>(16 * (p >> 2) + 4 * (p & 3) + u)));
            }
        }
        float scale = 1.f, unscale = 1.f;
        if constexpr (F16) {  // a power of two bringing the tile's largest magnitude into [0.5, 1)
            float mx = 0.f;
#pragma unroll
            for (int i = 0; i < 32; ++i) mx = fmaxf(mx, fmaxf(fabsf(x[i].x), fabsf(x[i].y)));
#pragma unroll
            for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            __syncthreads();  // the previous transform's readers of red are done
            if (lane == 0) red[warp] = mx;
            __syncthreads();
            mx = red[0];
#pragma unroll
            for (int w = 1; w < NT / 32; ++w) mx = fmaxf(mx, red[w]);
            if (mx > 0.f && isfinite(mx)) {
                int e;
                frexpf(mx, &e);
                scale = ldexpf(1.f, -e);
                unscale = ldexpf(1.f, e);
            }
        }
        // the stage-1 operand: per (a, m) one 16-byte vector of hi and one of lo
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int p = warp + 8 * q, a = p >> 2, m = p & 3;
            uint4 vh, vl;
            split2<F16>(x[4 * q + 0].x * scale, x[4 * q + 0].y * scale, vh.x, vl.x);
            split2<F16>(x[4 * q + 1].x * scale, x[4 * q + 1].y * scale, vh.y, vl.y);
            split2<F16>(x[4 * q + 2].x * scale, x[4 * q + 2].y * scale, vh.z, vl.z);
            split2<F16>(x[4 * q + 3].x * scale, x[4 * q + 3].y * scale, vh.w, vl.w);
            const uint32_t off = kmaj_off(a * CT + lane, 8 * m);
            *reinterpret_cast<uint4 *>(Ahi + off) = vh;
            *reinterpret_cast<uint4 *>(Alo + off) = vl;
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();
        if (threadIdx.x == 0) issue();
        ok = mbar_wait(sbar, phase);
        phase ^= 1;
        fence_after();
        if (ok) {
            // stage-1 epilogue: twiddle, split, and re-stage as the stage-2 operand
            // (rows (j, column), K digit a)
#pragma unroll
            for (int tt = 0; tt < 2; ++tt) {
                const int t = (warp >> 2) * 2 + tt;
                const int a = 4 * t + sp;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float v[16];
                    load_acc<F16>(tbase, sp, t, h, v);
#pragma unroll
                    for (int jl = 0; jl < RD / 2; ++jl) {
                        const int j = 8 * h + jl;
                        const int tw = (a * j) & (N - 1);
                        const float c = g_trig.c[tw], s = INV ? g_trig.s[tw] : -g_trig.s[tw];
                        const float re = v[2 * jl] * c - v[2 * jl + 1] * s, im = v[2 * jl] * s + v[2 * jl + 1] * c;
                        uint32_t hi, lo;
                        split2<F16>(re, im, hi, lo);
                        const uint32_t off = kmaj_off(j * CT + lane, 2 * a);
                        *reinterpret_cast<uint32_t *>(Ahi + off) = hi;
                        *reinterpret_cast<uint32_t *>(Alo + off) = lo;
                    }
                }
            }
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();
        ok = __syncthreads_and(ok);
        if (ok) {
            if (threadIdx.x == 0) issue();
            ok = mbar_wait(sbar, phase);
            phase ^= 1;
            fence_after();
            ok = __syncthreads_and(ok);
        }
        if (ok) {
            // stage-2 epilogue: row (j, column) holds the 16 outputs of digit o
#pragma unroll
            for (int tt = 0; tt < 2; ++tt) {
                const int t = (warp >> 2) * 2 + tt;
                const int j = 4 * t + sp;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float v[16];
                    load_acc<F16>(tbase, sp, t, h, v);
#pragma unroll
                    for (int ol = 0; ol < RD / 2; ++ol) {
                        const int o = 8 * h + ol;
                        const int row = INV ? j + RD * o : perm_slot<N>(j + RD * o);
                        dst[col + (size_t)row * H] = make_float2(v[2 * ol] * unscale, v[2 * ol + 1] * unscale);
                    }
                }
            }
            // the next transform's operand overwrites A and the accumulators
            fence_before();
            __syncthreads();
            fence_after();
        }
    }
    if (!ok && threadIdx.x == 0) {
        atomicAdd(&g_tc_timeouts, 1);
        // give a stalled MMA group a last bounded chance to drain before the
        // tensor memory is released
        mbar_wait(sbar, 0);
        mbar_wait(sbar, 1);
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(tmem_cols<F16>())
                     : "memory");
    }
}

template <bool INV, bool F16>
static cudaError_t launch(const float2 *s0, const float2 *s1, float2 *d0, float2 *d1, float2 *d2, int nrot,
                          cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        const cudaError_t e =
            cudaFuncSetAttribute(y_tc_kernel<INV, F16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
        if (e) return e;
        attr = true;
    }
    const dim3 grid(N * H / CT, nrot, INV ? 2 : 1);
    y_tc_kernel<INV, F16><<<grid, NT, SMEM, st>>>(s0, s1, d0, d1, d2);
    return cudaGetLastError();
}

}  // namespace tc

cudaError_t set_tc_attrs() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(tc::y_tc_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)tc::SMEM)))
        return e;
    if ((e = cudaFuncSetAttribute(tc::y_tc_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)tc::SMEM)))
        return e;
    if ((e = cudaFuncSetAttribute(tc::y_tc_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)tc::SMEM)))
        return e;
    return cudaFuncSetAttribute(tc::y_tc_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tc::SMEM);
}

cudaError_t run_yfwd_tc(int n, int prec, const float2 *Xa, float2 *X1, int nrot, cudaStream_t st) {
    if (n != tc::N || (prec != PREC_SPLIT_BF16 && prec != PREC_SPLIT_F16)) return cudaErrorInvalidValue;
    return prec == PREC_SPLIT_F16 ? tc::launch<false, true>(Xa, nullptr, X1, nullptr, nullptr, nrot, st)
                                  : tc::launch<false, false>(Xa, nullptr, X1, nullptr, nullptr, nrot, st);
}

cudaError_t run_yinv_tc(int n, int prec, const float2 *Y1, const float2 *Y2, float2 *ZS, float2 *ZGy, float2 *ZGz,
                        int nrot, cudaStream_t st) {
    if (n != tc::N || (prec != PREC_SPLIT_BF16 && prec != PREC_SPLIT_F16)) return cudaErrorInvalidValue;
    return prec == PREC_SPLIT_F16 ? tc::launch<true, true>(Y1, Y2, ZS, ZGy, ZGz, nrot, st)
                                  : tc::launch<true, false>(Y1, Y2, ZS, ZGy, ZGz, nrot, st);
}

int tc_timeouts(bool reset) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, tc::g_tc_timeouts, sizeof v) != cudaSuccess) return -1;
    if (reset) {
        const int z = 0;
        cudaMemcpyToSymbol(tc::g_tc_timeouts, &z, sizeof z);
    }
    return v;
}

// Never launched: its address names this file's device-code module, which
// hf_ctx_preload loads whole.
__global__ void module_anchor_tc_kernel() {}
const void *module_anchor_tc() { return (const void *)&module_anchor_tc_kernel; }

}  // namespace hf
