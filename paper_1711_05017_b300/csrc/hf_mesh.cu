// hf_mesh.cu -- the mesh descriptor of Eq. 2 (Section 2.3 "Skeletal
// Density", Section 3.1 "Preprocessing") on the N^3 nodes, for a closed
// triangle mesh with outward orientation:
//   W(p)   winding number: (1/4 pi) sum of the triangles' signed solid angles
//          (Eq. 2 with the inverse-square kernel; point membership)
//   xi(p)  signed distance to the surface, negative inside (the exact
//          point-triangle distance replaces the paper's OpenGL distance field)
//   rho(p) (1/4 pi) integral of exp(-(eta/|xi| - 1)^2 / 2 sigma^2) d gamma,
//          eta = |p - q|, d gamma the signed solid-angle element: the
//          inverse-square kernel weighted toward approximate nearest
//          boundary points, so high on the skeleton and -> W as sigma grows.
// The integral is a Riemann sum over triangles subdivided 4 ways at the edge
// midpoints until each piece subtends at most gamma_max (or depth dmax); a
// piece contributes the weight at its centroid times its exact solid angle.
// One thread per node, float64 throughout (an offline precompute; the
// membership sign and the subdivision decisions are then those of the FP64
// reference); the subdivision runs on an explicit depth-first stack.
#include <cuda_runtime.h>
#include <math.h>

#include "hf_internal.h"

namespace hf {

namespace {
constexpr int kMeshThreads = 128;
constexpr int kMaxDepth = 12;

struct D3 {
    double x, y, z;
};
__device__ __forceinline__ D3 sub(D3 a, D3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ double dot(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ D3 cross(D3 a, D3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ D3 mid(D3 a, D3 b) { return {0.5 * (a.x + b.x), 0.5 * (a.y + b.y), 0.5 * (a.z + b.z)}; }

// signed solid angle of (A, B, C) seen from p, van Oosterom and Strackee's
// formula; positive when p lies on the side opposite the normal (B-A)x(C-A)
__device__ __forceinline__ double solid_angle(D3 p, D3 A, D3 B, D3 C) {
    const D3 a = sub(A, p), b = sub(B, p), c = sub(C, p);
    const double la = sqrt(dot(a, a)), lb = sqrt(dot(b, b)), lc = sqrt(dot(c, c));
    const double num = dot(a, cross(b, c));
    const double den = la * lb * lc + dot(a, b) * lc + dot(a, c) * lb + dot(b, c) * la;
    return 2.0 * atan2(num, den);
}

// distance from p to triangle (A, B, C): face region by the barycentric
// coordinates of the projection, else the nearest of the three edges
__device__ __forceinline__ double tri_distance(D3 p, D3 A, D3 B, D3 C) {
    const D3 e0 = sub(B, A), e1 = sub(C, A), v = sub(p, A), nrm = cross(e0, e1);
    const double a00 = dot(e0, e0), a01 = dot(e0, e1), a11 = dot(e1, e1);
    const double b0 = dot(v, e0), b1 = dot(v, e1);
    const double det = a00 * a11 - a01 * a01;
    if (det > 0) {
        const double s = (a11 * b0 - a01 * b1) / det, t = (a00 * b1 - a01 * b0) / det;
        if (s >= 0 && t >= 0 && s + t <= 1) return fabs(dot(v, nrm)) / sqrt(dot(nrm, nrm));
    }
    const D3 P[3] = {A, B, C};
    double best = INFINITY;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const D3 X = P[k], Y = P[(k + 1) % 3];
        const D3 e = sub(Y, X), w = sub(p, X);
        double t = dot(w, e) / dot(e, e);
        t = t < 0 ? 0 : (t > 1 ? 1 : t);
        const D3 d = {w.x - t * e.x, w.y - t * e.y, w.z - t * e.z};
        best = fmin(best, sqrt(dot(d, d)));
    }
    return best;
}

__device__ __forceinline__ D3 vert(const double *V, int i) { return {__ldg(V + 3 * i), __ldg(V + 3 * i + 1), __ldg(V + 3 * i + 2)}; }

struct Piece {
    D3 a, b, c;
    int depth;
};

__global__ void __launch_bounds__(kMeshThreads) mesh_sdf_kernel(int n, const double *__restrict__ V,
                                                                const int *__restrict__ T, int nt, double sigma,
                                                                double gamma_max, int dmax, float *__restrict__ rho,
                                                                float *__restrict__ aux) {
    const size_t n3 = (size_t)n * n * n;
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n3) return;
    const double h = 2.0 / n;
    const int x = (int)(i % n), y = (int)((i / n) % n), z = (int)(i / ((size_t)n * n));
    const D3 p = {-1.0 + x * h, -1.0 + y * h, -1.0 + z * h};
    double w = 0, dist = INFINITY;
    for (int t = 0; t < nt; ++t) {
        const D3 A = vert(V, __ldg(T + 3 * t)), B = vert(V, __ldg(T + 3 * t + 1)), C = vert(V, __ldg(T + 3 * t + 2));
        w += solid_angle(p, A, B, C);
        dist = fmin(dist, tri_distance(p, A, B, C));
    }
    w /= 4.0 * 3.14159265358979323846;
    double acc = 0;
    if (dist > 1e-12) {
        const double inv2s2 = 0.5 / (sigma * sigma);
        Piece st[3 * kMaxDepth + 1];
        for (int t = 0; t < nt; ++t) {
            int sp = 0;
            st[sp++] = {vert(V, __ldg(T + 3 * t)), vert(V, __ldg(T + 3 * t + 1)), vert(V, __ldg(T + 3 * t + 2)), 0};
            while (sp > 0) {
                const Piece pc = st[--sp];
                const double om = solid_angle(p, pc.a, pc.b, pc.c);
                if (fabs(om) > gamma_max && pc.depth < dmax) {
                    const D3 ab = mid(pc.a, pc.b), bc = mid(pc.b, pc.c), ca = mid(pc.c, pc.a);
                    const int d = pc.depth + 1;
                    st[sp++] = {ab, bc, ca, d};
                    st[sp++] = {ca, bc, pc.c, d};
                    st[sp++] = {ab, pc.b, bc, d};
                    st[sp++] = {pc.a, ab, ca, d};
                } else {
                    const D3 q = {(pc.a.x + pc.b.x + pc.c.x) / 3, (pc.a.y + pc.b.y + pc.c.y) / 3,
                                  (pc.a.z + pc.b.z + pc.c.z) / 3};
                    const D3 dv = sub(q, p);
                    const double xr = sqrt(dot(dv, dv)) / dist - 1.0;
                    acc += exp(-xr * xr * inv2s2) * om;
                }
            }
        }
    }
    rho[i] = (float)(acc / (4.0 * 3.14159265358979323846));
    if (aux) {
        aux[i] = (float)w;
        aux[n3 + i] = (float)(w >= 0.5 ? -dist : dist);
    }
}
}  // namespace

cudaError_t run_mesh_sdf(int n, const double *V, const int *T, int nt, double sigma, double gamma_max, int dmax,
                         float *rho, float *aux, cudaStream_t st) {
    if (dmax > kMaxDepth) return cudaErrorInvalidValue;
    const size_t n3 = (size_t)n * n * n;
    const unsigned blocks = (unsigned)((n3 + kMeshThreads - 1) / kMeshThreads);
    mesh_sdf_kernel<<<blocks, kMeshThreads, 0, st>>>(n, V, T, nt, sigma, gamma_max, dmax, rho, aux);
    return cudaGetLastError();
}

}  // namespace hf
