// hf_dft.cuh -- register-level DFTs and the two-stage shared-memory FFT used
// by every pass of the field pipeline (the discrete transforms of Eqs. 7a/7b,
// Section 3.2, evaluated as mixed-radix Cooley-Tukey FFTs).
//
// Layout model.  A batch of M "lines" of length L lives in shared memory as
// float2; element j of line f is at base[f * ls + j * es].  A length
// L = R1 * R2 transform runs in two stages with a __syncthreads between them.
// Each thread owns R1 (or R2) elements in registers, transforms them with a
// fully unrolled register DFT and writes them back to the SAME slots it read,
// so no stage needs a second buffer:
//
//   forward  (natural order in, "digit-permuted" order out):
//     stage 1, items (f, n2):  slots n2 + R2*n1 (n1 < R1)  -> DFT_R1 over n1,
//              twiddle W_L^{n2 k1},  written back at n2 + R2*k1
//     stage 2, items (f, k1):  slots R2*k1 + n2 (n2 < R2) -> DFT_R2 over n2,
//              X[k1 + R1*k2] written at slot R2*k1 + k2
//   inverse  (digit-permuted in, natural out): the same two stages transposed.
//
// The frequency k sits at slot perm(k) = R2*(k % R1) + k / R1.
#pragma once
#include <cuda_runtime.h>
#include <type_traits>
#include <utility>

namespace hf {

// ------------------------------------------------------------------ complex
// Complex additions and subtractions are one paired FP32 instruction each
// (sm_100 and later: an add on a float2, every component rounded as the
// scalar operation, so the bits are those of two scalar adds; a + (-b) is
// a - b exactly, signed zeros included).
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
// the pair (u.x, u.y) times s, one paired instruction
__device__ __forceinline__ float2 cscale2(float2 u, float s) { return __fmul2_rn(u, make_float2(s, s)); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by i * s, as rounded products (never contracted into a following
// add), so that every kernel that applies the multiplier gives the same bits
__device__ __forceinline__ float2 cmul_is(float2 a, float s) { return make_float2(__fmul_rn(-a.y, s), __fmul_rn(a.x, s)); }

// ------------------------------------------------ compile-time trigonometry
// cos / sin of 2*pi*j/R in double, by octant reduction and Taylor series,
// evaluated by the compiler (all arguments are template constants).
namespace ct {
__host__ __device__ constexpr double sin_t(double x) {
    double x2 = x * x, term = x, sum = x;
    for (int k = 1; k < 14; ++k) { term *= -x2 / ((2.0 * k) * (2.0 * k + 1.0)); sum += term; }
    return sum;
}
__host__ __device__ constexpr double cos_t(double x) {
    double x2 = x * x, term = 1.0, sum = 1.0;
    for (int k = 1; k < 14; ++k) { term *= -x2 / ((2.0 * k - 1.0) * (2.0 * k)); sum += term; }
    return sum;
}
constexpr double kQuarterPi = 0.78539816339744830961566084581987572;
// cos (which = 0) or sin (which = 1) of 2 pi j / R
__host__ __device__ constexpr double trig(long j, long R, int which) {
    long jj = ((j % R) + R) % R;
    long num = 8 * jj;          // angle = (pi/4) * num / R
    long o = num / R;           // octant 0..7
    long rem = num - o * R;     // angle within the octant = (pi/4) * rem / R
    double phi = kQuarterPi * (double)rem / (double)R;
    double psi = kQuarterPi * (double)(R - rem) / (double)R;  // pi/4 - phi
    double c = 0, s = 0;
    switch (o & 3) {
        case 0: c = cos_t(phi); s = sin_t(phi); break;
        case 1: c = sin_t(psi); s = cos_t(psi); break;
        case 2: c = -sin_t(phi); s = cos_t(phi); break;
        default: c = -cos_t(psi); s = sin_t(psi); break;
    }
    if (o >= 4) { c = -c; s = -s; }
    return which == 0 ? c : s;
}
}  // namespace ct

// ---------------------------------------------------------------- twiddles
struct cf2 {
    float x, y;
};
template <int L>
struct TwTab {
    cf2 v[L];
};
template <int L>
constexpr TwTab<L> make_tw() {
    TwTab<L> t{};
    for (int j = 0; j < L; ++j) {
        t.v[j].x = (float)ct::trig(j, L, 0);
        t.v[j].y = (float)(-ct::trig(j, L, 1));  // exp(-2 pi i j / L)
    }
    return t;
}
template <int L>
__device__ const TwTab<L> g_tw = make_tw<L>();
// the same table in constant memory, for twiddles read at a warp-uniform
// index (served by the constant cache, off the shared-memory pipe)
template <int L>
__constant__ TwTab<L> c_tw = make_tw<L>();
template <int L>
__device__ __forceinline__ float2 tw_uniform(int j) {
    const cf2 t = c_tw<L>.v[j];
    return make_float2(t.x, t.y);
}
// twiddle j of length L: from constant memory when the caller's index is
// warp-uniform (UNIFORM), else from the shared copy tw
template <int L, bool UNIFORM>
__device__ __forceinline__ float2 tw_pick(const float2 *tw, int j) {
    if constexpr (UNIFORM) return tw_uniform<L>(j);
    else return tw[j];
}


template <int I, int E, class F>
__device__ __forceinline__ void static_for(F &&f) {
    if constexpr (I < E) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, E>(f);
    }
}

// x * exp(DIR * 2 pi i * M / R), M and R compile-time
template <int M, int R, int DIR>
__device__ __forceinline__ float2 twiddle_c(float2 x) {
    constexpr int m = ((M % R) + R) % R;
    if constexpr (m == 0) {
        return x;
    } else if constexpr ((8 * m) % R == 0) {
        constexpr int o = (8 * m / R) * (DIR > 0 ? 1 : 7) % 8;  // octant of DIR * angle
        constexpr float r = 0.70710678118654752440f;
        if constexpr (o == 2) return make_float2(-x.y, x.x);       // * i
        else if constexpr (o == 4) return make_float2(-x.x, -x.y);  // * -1
        else if constexpr (o == 6) return make_float2(x.y, -x.x);   // * -i
        else if constexpr (o == 1) return cscale2(make_float2(x.x - x.y, x.x + x.y), r);
        else if constexpr (o == 3) return cscale2(make_float2(-(x.x + x.y), x.x - x.y), r);
        else if constexpr (o == 5) return cscale2(make_float2(x.y - x.x, -(x.x + x.y)), r);
        else return cscale2(make_float2(x.x + x.y, x.y - x.x), r);  // o == 7
    } else {
        constexpr float c = (float)ct::trig(m, R, 0);
        constexpr float s = (float)(DIR * ct::trig(m, R, 1));
        return make_float2(fmaf(x.x, c, -x.y * s), fmaf(x.x, s, x.y * c));
    }
}

// ----------------------------------------------------------- register DFTs
// In-place natural-order DFT of R registers:
//   X[k] = sum_j x[j] exp(DIR * 2 pi i j k / R)   (DIR = -1 forward, +1 inverse)
template <int R, int DIR>
struct RegDFT;

template <int DIR>
struct RegDFT<1, DIR> {
    __device__ __forceinline__ static void run(float2 *) {}
};

template <int DIR>
struct RegDFT<2, DIR> {
    __device__ __forceinline__ static void run(float2 *x) {
        float2 a = x[0], b = x[1];
        x[0] = cadd(a, b);
        x[1] = csub(a, b);
    }
};

template <int DIR>
struct RegDFT<3, DIR> {
    __device__ __forceinline__ static void run(float2 *x) {
        constexpr float s3 = 0.86602540378443864676f * (float)DIR;
        float2 t = cadd(x[1], x[2]), d = csub(x[1], x[2]);
        float2 m = __ffma2_rn(make_float2(-0.5f, -0.5f), t, x[0]);
        float2 r = make_float2(-d.y * s3, d.x * s3);  // i * DIR * (sqrt3/2) * d
        x[0] = cadd(x[0], t);
        x[1] = cadd(m, r);
        x[2] = csub(m, r);
    }
};

template <int DIR>
struct RegDFT<4, DIR> {
    __device__ __forceinline__ static void run(float2 *x) {
        float2 s02 = cadd(x[0], x[2]), d02 = csub(x[0], x[2]);
        float2 s13 = cadd(x[1], x[3]), d13 = csub(x[1], x[3]);
        x[0] = cadd(s02, s13);
        x[2] = csub(s02, s13);
        // d02 +- W d13 with W = DIR * i, as scalar adds (the swapped pair
        // would cost moves): the same sums as adding (-d13.y, d13.x) or
        // (d13.y, -d13.x)
        if constexpr (DIR > 0) {
            x[1] = make_float2(d02.x - d13.y, d02.y + d13.x);
            x[3] = make_float2(d02.x + d13.y, d02.y - d13.x);
        } else {
            x[1] = make_float2(d02.x + d13.y, d02.y - d13.x);
            x[3] = make_float2(d02.x - d13.y, d02.y + d13.x);
        }
    }
};

// Composite R = P * Q, decimation in time:
//   Y_p = DFT_Q(x[p], x[p+P], ...),  Y_p[kq] *= W_R^{p kq},  X[kq + Q kp] = DFT_P over p
template <int R, int DIR>
struct RegDFT {
    static constexpr int P = (R % 4 == 0) ? 4 : (R % 2 == 0) ? 2 : 3;
    static constexpr int Q = R / P;
    static_assert(P * Q == R && Q > 1, "unsupported register DFT length");
    __device__ __forceinline__ static void run(float2 *x) {
        float2 y[P][Q];
        static_for<0, P>([&](auto pp) {
            constexpr int p = decltype(pp)::value;
            static_for<0, Q>([&](auto qq) {
                constexpr int q = decltype(qq)::value;
                y[p][q] = x[p + P * q];
            });
            RegDFT<Q, DIR>::run(y[p]);
            static_for<0, Q>([&](auto kk) {
                constexpr int kq = decltype(kk)::value;
                y[p][kq] = twiddle_c<p * kq, R, DIR>(y[p][kq]);
            });
        });
        static_for<0, Q>([&](auto kk) {
            constexpr int kq = decltype(kk)::value;
            float2 z[P];
            static_for<0, P>([&](auto pp) { z[decltype(pp)::value] = y[decltype(pp)::value][kq]; });
            RegDFT<P, DIR>::run(z);
            static_for<0, P>([&](auto pp) {
                constexpr int kp = decltype(pp)::value;
                x[kq + Q * kp] = z[kp];
            });
        });
    }
};

// ------------------------------------------------ factorisation of lengths
// L = R1 * R2 for the two shared-memory stages.
template <int L>
struct Fact;
template <> struct Fact<16> { static constexpr int R1 = 4, R2 = 4; };
template <> struct Fact<32> { static constexpr int R1 = 8, R2 = 4; };
template <> struct Fact<48> { static constexpr int R1 = 8, R2 = 6; };
template <> struct Fact<64> { static constexpr int R1 = 8, R2 = 8; };
template <> struct Fact<96> { static constexpr int R1 = 12, R2 = 8; };
template <> struct Fact<128> { static constexpr int R1 = 16, R2 = 8; };
template <> struct Fact<256> { static constexpr int R1 = 16, R2 = 16; };

// slot of frequency k in a digit-permuted line of length L
template <int L>
__device__ __forceinline__ int perm_slot(int k) {
    return Fact<L>::R2 * (k % Fact<L>::R1) + k / Fact<L>::R1;
}
// frequency held by slot s
template <int L>
__device__ __forceinline__ int slot_freq(int s) {
    return s / Fact<L>::R2 + Fact<L>::R1 * (s % Fact<L>::R2);
}

// ------------------------------------------------ two-stage batched FFT
// tw[j] = exp(-2 pi i j / L), j < L (forward sign), in shared memory; where
// M is a multiple of 32 a warp's twiddle index is uniform and the constant-
// memory copy of the same table is read instead.
// M lines; element j of line f at base[f * LS + j * ES]; NT threads.  All
// sizes are compile-time so every index is a multiply-shift.  All threads of
// the block must call; ends with __syncthreads.
template <int L, int DIR, int M, int ES, int LS, int NT>
__device__ __forceinline__ void fft_lines(float2 *base, const float2 *tw) {
    constexpr int R1 = Fact<L>::R1, R2 = Fact<L>::R2;
    if constexpr (DIR < 0) {
        // stage 1: items (f, n2)
#pragma unroll 1
        for (int w = threadIdx.x; w < M * R2; w += NT) {
            const int f = w % M, n2 = w / M;
            float2 *p = base + f * LS + n2 * ES;
            float2 v[R1];
#pragma unroll
            for (int n1 = 0; n1 < R1; ++n1) v[n1] = p[n1 * R2 * ES];
            RegDFT<R1, -1>::run(v);
#pragma unroll
            for (int k1 = 1; k1 < R1; ++k1) v[k1] = cmul(v[k1], tw_pick<L, M % 32 == 0>(tw, n2 * k1));
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1) p[k1 * R2 * ES] = v[k1];
        }
        __syncthreads();
        // stage 2: items (f, k1)
#pragma unroll 1
        for (int w = threadIdx.x; w < M * R1; w += NT) {
            const int f = w % M, k1 = w / M;
            float2 *p = base + f * LS + (R2 * k1) * ES;
            float2 v[R2];
#pragma unroll
            for (int n2 = 0; n2 < R2; ++n2) v[n2] = p[n2 * ES];
            RegDFT<R2, -1>::run(v);
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) p[k2 * ES] = v[k2];
        }
        __syncthreads();
    } else {
        // stage 1: items (f, k1): slots R2*k1 + k2 hold X[k1 + R1*k2]
#pragma unroll 1
        for (int w = threadIdx.x; w < M * R1; w += NT) {
            const int f = w % M, k1 = w / M;
            float2 *p = base + f * LS + (R2 * k1) * ES;
            float2 v[R2];
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) v[k2] = p[k2 * ES];
            RegDFT<R2, +1>::run(v);
#pragma unroll
            for (int n2 = 1; n2 < R2; ++n2) v[n2] = cmulc(v[n2], tw_pick<L, M % 32 == 0>(tw, n2 * k1));
#pragma unroll
            for (int n2 = 0; n2 < R2; ++n2) p[n2 * ES] = v[n2];
        }
        __syncthreads();
        // stage 2: items (f, n2)
#pragma unroll 1
        for (int w = threadIdx.x; w < M * R2; w += NT) {
            const int f = w % M, n2 = w / M;
            float2 *p = base + f * LS + n2 * ES;
            float2 v[R1];
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1) v[k1] = p[k1 * R2 * ES];
            RegDFT<R1, +1>::run(v);
#pragma unroll
            for (int n1 = 0; n1 < R1; ++n1) p[n1 * R2 * ES] = v[n1];
        }
        __syncthreads();
    }
}

}  // namespace hf
