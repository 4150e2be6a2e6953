// hf_spec.cuh -- device helpers of the frequency-domain rotation (Section
// 3.2, step 1): the moving part's centred spectrum table, rotated
// coordinates in double-float arithmetic, slot order of the x half spectrum.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "hf_dft.cuh"

namespace hf {

// x slot of half-spectrum index k in [0, N/2]
template <int N>
__device__ __forceinline__ int xslot(int k) {
    return k == N / 2 ? N / 2 : perm_slot<N / 2>(k);
}

// The rotated moving spectrum is read off a moving part's centred table
// (os N per axis, full cube, natural order) by periodic trilinear
// interpolation at os R^T k~ (Section 3.2, step 1).  The coordinate is
// summed in double-float arithmetic (exact products, compensated sums) so
// that the fractional weights carry the rotation to ~1e-12 at any table
// size.
struct SpecSrc {
    const float2 *table;
    int np;  // os * N
    int os;
    // the same table as stacked, wrap-padded (np+1)^2 slices of a float2
    // gather texture, sc slices per texture row (read by the field build)
    cudaTextureObject_t tex = 0;
    int sc = 0;
};

// slices per row of a table texture of np^3 cells
__host__ __device__ __forceinline__ int table_tex_sc(int np) { return np >= 128 ? 16 : 8; }

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// floor and fraction of r0 k0 + r1 k1 + r2 k2 (integer k), accurate
__device__ __forceinline__ void rot_coord(float r0, float r1, float r2, float k0, float k1, float k2, int &i0,
                                          float &fr) {
    const float p0 = r0 * k0, p1 = r1 * k1, p2 = r2 * k2;
    const float e0 = fmaf(r0, k0, -p0), e1 = fmaf(r1, k1, -p1), e2 = fmaf(r2, k2, -p2);
    float s01, t01, s, t;
    two_sum(p0, p1, s01, t01);
    two_sum(s01, p2, s, t);
    const float corr = ((t01 + t) + (e0 + e1)) + e2;
    const float fl = floorf(s);
    fr = (s - fl) + corr;  // s - fl is exact
    i0 = (int)fl;
    if (fr < 0.f) {
        fr += 1.f;
        --i0;
    } else if (fr >= 1.f) {
        fr -= 1.f;
        ++i0;
    }
}

// periodic wrap of a table index (np is a power of two except at 96)
__device__ __forceinline__ int table_wrap(int v, int np) {
    if ((np & (np - 1)) == 0) return v & (np - 1);
    const int r = v % np;
    return r < 0 ? r + np : r;
}

}  // namespace hf
