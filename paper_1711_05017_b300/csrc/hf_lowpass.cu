// hf_lowpass.cu -- energy, force and torque at single poses from truncated
// spectra (Section 4.2, "Truncated Inverse FFT", with the low-pass filtering
// of Section 3.3): for a pose (R, t), only the modes |k~_a| <= K of
//   S(k) = (h^3/N^3) rho1^(k) conj(B(k)),
//   B(k) = (-1)^(kx+ky+kz) trilinear(table, os R^T k~)   (Section 3.2, step 1)
// are kept, and the inverse transform is summed at the one translation t:
//   E   = sum Re S e^{i pi k~.t}                 (omega = k~/2 since N h = 2)
//   F_d = sum pi k~_d Im(S e^{i pi k~.t})        (= -d E / d t_d, Eq. 6a)
//   T_a = -d E / d theta_a for R -> exp(theta [e_a]x) R, through the
//         interpolant: d(os R^T k~)/d theta_a = -os R^T (e_a x k~).
// Each pose is spread over up to kLowpassMaxSplit CTAs of 256 threads; each
// thread takes modes in turn and accumulates in float64 (the sum of (2K+1)^3
// terms cancels heavily); the last CTA of a pose adds the CTAs' partial sums
// in a fixed order.  The phases come from per-axis float64 tables.
#include <cuda_runtime.h>
#include <math.h>

#include "hf_internal.h"
#include "hf_spec.cuh"

namespace hf {

namespace {
constexpr int kLpThreads = 256;

// trilinear value and index-space gradient of the complex table at the
// coordinate (i + w) per axis
__device__ __forceinline__ float2 table_trilinear(const SpecSrc &src, const int i[3], const float w[3],
                                                  float2 g[3]) {
    const int np = src.np;
    const int x0 = table_wrap(i[0], np), x1 = table_wrap(i[0] + 1, np);
    const int y0 = table_wrap(i[1], np), y1 = table_wrap(i[1] + 1, np);
    const float2 *p0 = src.table + (size_t)table_wrap(i[2], np) * np * np;
    const float2 *p1 = src.table + (size_t)table_wrap(i[2] + 1, np) * np * np;
    float2 c[2][2][2];
    c[0][0][0] = __ldg(p0 + (size_t)y0 * np + x0);
    c[0][0][1] = __ldg(p0 + (size_t)y0 * np + x1);
    c[0][1][0] = __ldg(p0 + (size_t)y1 * np + x0);
    c[0][1][1] = __ldg(p0 + (size_t)y1 * np + x1);
    c[1][0][0] = __ldg(p1 + (size_t)y0 * np + x0);
    c[1][0][1] = __ldg(p1 + (size_t)y0 * np + x1);
    c[1][1][0] = __ldg(p1 + (size_t)y1 * np + x0);
    c[1][1][1] = __ldg(p1 + (size_t)y1 * np + x1);
    float2 v = make_float2(0.f, 0.f);
    g[0] = g[1] = g[2] = make_float2(0.f, 0.f);
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                const float wx = dx ? w[0] : 1.f - w[0], wy = dy ? w[1] : 1.f - w[1], wz = dz ? w[2] : 1.f - w[2];
                const float sx = dx ? 1.f : -1.f, sy = dy ? 1.f : -1.f, sz = dz ? 1.f : -1.f;
                const float2 cc = c[dz][dy][dx];
                const float a = wx * wy * wz, bx = sx * wy * wz, by = wx * sy * wz, bz = wx * wy * sz;
                v.x = fmaf(a, cc.x, v.x);
                v.y = fmaf(a, cc.y, v.y);
                g[0].x = fmaf(bx, cc.x, g[0].x);
                g[0].y = fmaf(bx, cc.y, g[0].y);
                g[1].x = fmaf(by, cc.x, g[1].x);
                g[1].y = fmaf(by, cc.y, g[1].y);
                g[2].x = fmaf(bz, cc.x, g[2].x);
                g[2].y = fmaf(bz, cc.y, g[2].y);
            }
    return v;
}

// pose q = (w, x, y, z) -> float32 rotation matrix through float64 (as the
// host does for field sets)
__device__ __forceinline__ void quat_rot9(const float *q4, float *R) {
    const double w0 = q4[0], x0 = q4[1], y0 = q4[2], z0 = q4[3];
    const double nn = sqrt(w0 * w0 + x0 * x0 + y0 * y0 + z0 * z0);
    const double w = w0 / nn, x = x0 / nn, y = y0 / nn, z = z0 / nn;
    R[0] = (float)(1 - 2 * (y * y + z * z));
    R[1] = (float)(2 * (x * y - w * z));
    R[2] = (float)(2 * (x * z + w * y));
    R[3] = (float)(2 * (x * y + w * z));
    R[4] = (float)(1 - 2 * (x * x + z * z));
    R[5] = (float)(2 * (y * z - w * x));
    R[6] = (float)(2 * (x * z - w * y));
    R[7] = (float)(2 * (y * z + w * x));
    R[8] = (float)(1 - 2 * (x * x + y * y));
}

template <int N>
__global__ void __launch_bounds__(kLpThreads) lowpass_kernel(const float2 *__restrict__ spec1, SpecSrc tab, int K,
                                                             const float *__restrict__ tq, LowpassPose one,
                                                             double *__restrict__ part, unsigned *__restrict__ count,
                                                             float *__restrict__ out) {
    constexpr int H = N / 2 + 1;
    constexpr double kPiD = 3.14159265358979323846;
    extern __shared__ double2 ph[];  // per-axis phases e^{i pi k t_a}, [3][2K+1], float64
    __shared__ double red[kLpThreads / 32][7];
    __shared__ bool last;
    const int q = blockIdx.y, split = gridDim.x;
    float R[9], t[3];
    if (tq) {
        const float *p = tq + 7 * (size_t)q;
        quat_rot9(p + 3, R);
        t[0] = p[0];
        t[1] = p[1];
        t[2] = p[2];
    } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) R[k] = one.R[k];
        t[0] = one.t[0];
        t[1] = one.t[1];
        t[2] = one.t[2];
    }
    const int side = 2 * K + 1, modes = side * side * side;
    for (int i = threadIdx.x; i < 3 * side; i += kLpThreads) {
        double sp, cp;
        sincospi((double)(i % side - K) * (double)t[i / side], &sp, &cp);
        ph[i] = make_double2(cp, sp);
    }
    __syncthreads();
    const float os = (float)tab.os;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int m = blockIdx.x * kLpThreads + threadIdx.x; m < modes; m += split * kLpThreads) {
        const int ix = m % side, iy = (m / side) % side, iz = m / (side * side);
        const int kx = ix - K, ky = iy - K, kz = iz - K;
        // stationary coefficient (h^3/N^3) rho1^(k): slot-order half spectrum,
        // negative kx by Hermitian symmetry
        const int ax = kx < 0 ? -kx : kx, sy = kx < 0 ? -ky : ky, sz = kx < 0 ? -kz : kz;
        float2 a1 = __ldg(spec1 + ((size_t)perm_slot<N>((sz + N) % N) * N + perm_slot<N>((sy + N) % N)) * H +
                          xslot<N>(ax));
        if (kx < 0) a1.y = -a1.y;
        if ((kx + ky + kz) & 1) a1 = make_float2(-a1.x, -a1.y);  // the table's centring sign, folded in
        int ii[3];
        float w[3];
        const float kf[3] = {os * kx, os * ky, os * kz};
#pragma unroll
        for (int a = 0; a < 3; ++a) rot_coord(R[a], R[3 + a], R[6 + a], kf[0], kf[1], kf[2], ii[a], w[a]);
        float2 g[3];
        const float2 b = table_trilinear(tab, ii, w, g);
        // phase e^{i pi k.t} = product of the three axis phases
        const double2 px = ph[ix], py = ph[side + iy], pz = ph[2 * side + iz];
        const double qxr = px.x * py.x - px.y * py.y, qxi = px.x * py.y + px.y * py.x;
        const double cp = qxr * pz.x - qxi * pz.y, sp = qxr * pz.y + qxi * pz.x;
        // term = a1 conj(b) e^{i phi}
        const double pr = (double)a1.x * b.x + (double)a1.y * b.y, pi_ = (double)a1.y * b.x - (double)a1.x * b.y;
        const double tr = pr * cp - pi_ * sp, ti = pr * sp + pi_ * cp;
        acc[0] += tr;
        acc[1] += kPiD * kx * ti;
        acc[2] += kPiD * ky * ti;
        acc[3] += kPiD * kz * ti;
        // torque: d b / d theta_a = grad . v_a,  v_a = -os R^T (e_a x k)
        const float ek[3][3] = {{0.f, -(float)kz, (float)ky}, {(float)kz, 0.f, -(float)kx}, {-(float)ky, (float)kx, 0.f}};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float2 db = make_float2(0.f, 0.f);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float vc = -os * (R[c] * ek[a][0] + R[3 + c] * ek[a][1] + R[6 + c] * ek[a][2]);
                db.x = fmaf(g[c].x, vc, db.x);
                db.y = fmaf(g[c].y, vc, db.y);
            }
            const double qr = (double)a1.x * db.x + (double)a1.y * db.y,
                         qi = (double)a1.y * db.x - (double)a1.x * db.y;
            acc[4 + a] -= qr * cp - qi * sp;
        }
    }
#pragma unroll
    for (int i = 0; i < 7; ++i)
#pragma unroll
        for (int o = 16; o; o >>= 1) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < 7; ++i) red[warp][i] = acc[i];
    __syncthreads();
    // this block's partial sums; the last block of the pose adds all partials
    // in block order (deterministic) and resets the pose's counter
    double *mine = part + ((size_t)q * split + blockIdx.x) * 7;
    if (threadIdx.x < 7) {
        double s = 0;
        for (int w2 = 0; w2 < kLpThreads / 32; ++w2) s += red[w2][threadIdx.x];
        mine[threadIdx.x] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(count + q, 1u) == (unsigned)split - 1;
    __syncthreads();
    if (last && threadIdx.x < 7) {
        __threadfence();
        const volatile double *all = part + (size_t)q * split * 7;
        double s = 0;
        for (int b2 = 0; b2 < split; ++b2) s += all[b2 * 7 + threadIdx.x];
        out[7 * (size_t)q + threadIdx.x] = (float)s;
        if (threadIdx.x == 0) count[q] = 0;
    }
}
}  // namespace

#define HF_DISPATCH_LP(n, call)                             \
    switch (n) {                                            \
        case 32: { constexpr int NN = 32; call; break; }    \
        case 64: { constexpr int NN = 64; call; break; }    \
        case 96: { constexpr int NN = 96; call; break; }    \
        case 128: { constexpr int NN = 128; call; break; }  \
        case 256: { constexpr int NN = 256; call; break; }  \
        default: return cudaErrorInvalidValue;              \
    }

int lowpass_split(int K) {
    const long modes = (long)(2 * K + 1) * (2 * K + 1) * (2 * K + 1);
    const long b = (modes + kLpThreads - 1) / kLpThreads;
    return (int)(b < kLowpassMaxSplit ? b : kLowpassMaxSplit);
}

cudaError_t run_lowpass(int n, const float2 *spec1, const float2 *table, int os, int K, const float *d_tq, int Q,
                        const LowpassPose *one, double *part, unsigned *count, float *out, cudaStream_t st) {
    if (Q <= 0) return cudaSuccess;
    const SpecSrc tab{table, os * n, os};
    const LowpassPose p = one ? *one : LowpassPose{};
    const dim3 grid(lowpass_split(K), Q);
    const size_t sm = sizeof(double2) * 3 * (2 * K + 1);
    HF_DISPATCH_LP(n, (lowpass_kernel<NN><<<grid, kLpThreads, sm, st>>>(spec1, tab, K, one ? nullptr : d_tq, p, part,
                                                                       count, out)));
    return cudaGetLastError();
}

}  // namespace hf
