// hf_sample.cuh -- periodic trilinear sampling of a density grid at rotated
// node positions (Section 2.4, motion decomposition: rho(R^T (p - t)) ).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace hf {

template <int N>
__device__ __forceinline__ int wrapN(int i) {
    if constexpr ((N & (N - 1)) == 0) return i & (N - 1);
    else { int r = i % N; return r < 0 ? r + N : r; }
}

// periodic trilinear sample of rho at centred index coordinates v (node N/2 = origin)
template <int N>
__device__ __forceinline__ float trilinear_c(const float *__restrict__ rho, float vx, float vy, float vz) {
    const float fx = floorf(vx), fy = floorf(vy), fz = floorf(vz);
    const float ax = vx - fx, ay = vy - fy, az = vz - fz;
    const int x0 = wrapN<N>((int)fx + N / 2), y0 = wrapN<N>((int)fy + N / 2), z0 = wrapN<N>((int)fz + N / 2);
    const int x1 = wrapN<N>(x0 + 1), y1 = wrapN<N>(y0 + 1), z1 = wrapN<N>(z0 + 1);
    const float *r00 = rho + ((size_t)z0 * N + y0) * N, *r01 = rho + ((size_t)z0 * N + y1) * N;
    const float *r10 = rho + ((size_t)z1 * N + y0) * N, *r11 = rho + ((size_t)z1 * N + y1) * N;
    float c00 = fmaf(ax, __ldg(r00 + x1) - __ldg(r00 + x0), __ldg(r00 + x0));
    float c01 = fmaf(ax, __ldg(r01 + x1) - __ldg(r01 + x0), __ldg(r01 + x0));
    float c10 = fmaf(ax, __ldg(r10 + x1) - __ldg(r10 + x0), __ldg(r10 + x0));
    float c11 = fmaf(ax, __ldg(r11 + x1) - __ldg(r11 + x0), __ldg(r11 + x0));
    float c0 = fmaf(ay, c01 - c00, c00), c1 = fmaf(ay, c11 - c10, c10);
    return fmaf(az, c1 - c0, c0);
}

}  // namespace hf
