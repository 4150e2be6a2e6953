/*
 * hf_oracle.c -- plain FP64 CPU oracle for the skeletal-density correlation
 * path of Behandish & Ilies, "Haptic Assembly Using Skeletal Densities and
 * Fourier Transforms" (ASME JCISE 16(2), 2016).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, call or
 * execute this file; only the test-suite, the package smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code, header, table or
 * constant with the CUDA library.
 *
 * Every routine is the plain definition written out, in double precision,
 * with at most an OpenMP "parallel for" over independent outer iterations.
 * There is no blocking, fusion or reordering beyond what the definition
 * states.
 *
 * Conventions (readings of passages the paper leaves open):
 *   grid      N^3 nodes on the periodic box [-1,1)^3, h = 2/N,
 *             node x_n = -1 + n*h, arrays indexed [z][y][x] (x fastest).
 *   lags      translation t_j = j*h, j wrapped to the torus; lag 0 at index 0.
 *   DFT       unscaled forward sum with e^{-2 pi i k n / N}; inverse carries
 *             1/N^3 (Eqs. 7a/7b up to their "constant factor").
 *   energy    E = +f_SC, the Riemann sum of Eq. 1 with volume element h^3.
 *   force     F = -grad_t E via the multiplier 2 pi i omega of Eq. 6a,
 *             omega = k~/(N h), k~ signed, Nyquist multiplier set to 0.
 *   torque    T = -grad_theta E by least squares over the 6 nearest sampled
 *             rotations (left perturbation R_j = exp([d theta]x) R_i).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

static const double PI = 3.14159265358979323846264338327950288;

static int wrap(long i, int n) {
    long r = i % n;
    return (int)(r < 0 ? r + n : r);
}

static long idx3(int n, int z, int y, int x) {
    return ((long)z * n + y) * n + x;
}

/* ------------------------------------------------------------------ */
/* Skeletal density (stand-in for the SDF of Eq. 2, Section 2.3):       */
/* a sum of isotropic Gaussian kernels centred on skeleton samples,     */
/* peak amplitude a_i, truncated at |r| <= cutoff*sigma_i, distances    */
/* measured by the minimum image on the torus of period 2.             */
/* ------------------------------------------------------------------ */
void or_splat(int n, int npts, const double *pts, const double *sigma,
              const double *amp, double cutoff, double *rho)
{
    const double h = 2.0 / n;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < n; ++z) {
        for (int y = 0; y < n; ++y) {
            for (int x = 0; x < n; ++x) {
                const double p[3] = {-1.0 + x * h, -1.0 + y * h, -1.0 + z * h};
                double acc = 0.0;
                for (int i = 0; i < npts; ++i) {
                    double r2 = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        double d = p[a] - pts[3 * i + a];
                        d -= 2.0 * nearbyint(d / 2.0); /* minimum image */
                        r2 += d * d;
                    }
                    const double s = sigma[i];
                    if (r2 <= cutoff * cutoff * s * s)
                        acc += (amp ? amp[i] : 1.0) * exp(-r2 / (2.0 * s * s));
                }
                rho[idx3(n, z, y, x)] = acc;
            }
        }
    }
}

/* Unit quaternion (w,x,y,z) -> proper orthogonal 3x3 matrix, row-major. */
void or_quat_to_rot(const double *q_in, double *R)
{
    double nrm = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] +
                      q_in[2] * q_in[2] + q_in[3] * q_in[3]);
    double w = q_in[0] / nrm, x = q_in[1] / nrm, y = q_in[2] / nrm, z = q_in[3] / nrm;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* Periodic trilinear sample of a grid at continuous index coordinates u. */
static double trilinear(int n, const double *g, const double u[3])
{
    long i0[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double fl = floor(u[a]);
        i0[a] = (long)fl;
        f[a] = u[a] - fl;
    }
    double acc = 0.0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                double w = (dx ? f[0] : 1 - f[0]) * (dy ? f[1] : 1 - f[1]) *
                           (dz ? f[2] : 1 - f[2]);
                acc += w * g[idx3(n, wrap(i0[2] + dz, n), wrap(i0[1] + dy, n),
                                  wrap(i0[0] + dx, n))];
            }
    return acc;
}

/* ------------------------------------------------------------------ */
/* Rotated moving density, Section 2.4 "Motion Decomposition":          */
/*   rho2^R(p) = rho2(R^T p), sampled at the nodes by periodic          */
/*   trilinear interpolation of the rho2 grid.                          */
/* ------------------------------------------------------------------ */
void or_resample(int n, const double *rho, const double *R, double *out)
{
    const double h = 2.0 / n;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < n; ++z)
        for (int y = 0; y < n; ++y)
            for (int x = 0; x < n; ++x) {
                const double p[3] = {-1.0 + x * h, -1.0 + y * h, -1.0 + z * h};
                double u[3];
                for (int a = 0; a < 3; ++a) {
                    /* (R^T p)_a = sum_b R[b][a] p_b, then to index units */
                    double q = R[0 * 3 + a] * p[0] + R[1 * 3 + a] * p[1] + R[2 * 3 + a] * p[2];
                    u[a] = (q + 1.0) / h;
                }
                out[idx3(n, z, y, x)] = trilinear(n, rho, u);
            }
}

/* ------------------------------------------------------------------ */
/* Discrete Fourier transform, Eqs. 7a/7b and Section 3.2:              */
/* recursive mixed-radix Cooley-Tukey, decimation in time.  A length    */
/* n = p*m splits into p interleaved subsequences of length m whose     */
/* transforms Y_r combine as X[k + s*m] = sum_r W_n^{r(k+s*m)} Y_r[k].  */
/* A prime length falls back to the direct DFT sum.                     */
/* sign = -1 forward, +1 inverse (unscaled both ways).                  */
/* ------------------------------------------------------------------ */
static int smallest_factor(int n)
{
    for (int p = 2; p * p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

static void fft_rec(int n, const cplx *in, long stride, cplx *out, int sign)
{
    if (n == 1) { out[0] = in[0]; return; }
    int p = smallest_factor(n);
    if (p == n) { /* direct DFT of a prime length */
        for (int k = 0; k < n; ++k) {
            cplx acc = 0;
            for (int j = 0; j < n; ++j)
                acc += in[j * stride] * cexp(sign * 2.0 * PI * I * (double)((long)j * k % n) / n);
            out[k] = acc;
        }
        return;
    }
    int m = n / p;
    cplx *sub = malloc(sizeof(cplx) * n);
    for (int r = 0; r < p; ++r)
        fft_rec(m, in + r * stride, stride * p, sub + r * m, sign);
    for (int k = 0; k < m; ++k)
        for (int s = 0; s < p; ++s) {
            int kk = k + s * m;
            cplx acc = 0;
            for (int r = 0; r < p; ++r)
                acc += sub[r * m + k] * cexp(sign * 2.0 * PI * I * (double)((long)r * kk % n) / n);
            out[kk] = acc;
        }
    free(sub);
}

void or_fft1d(int n, const double *in_ri, double *out_ri, int sign)
{
    fft_rec(n, (const cplx *)in_ri, 1, (cplx *)out_ri, sign);
}

/* Full complex 3D DFT of an n^3 array ([z][y][x]), one axis at a time. */
void or_fft3d(int n, double *data_ri, int sign)
{
    cplx *a = (cplx *)data_ri;
    for (int axis = 0; axis < 3; ++axis) {
        long st = axis == 0 ? 1 : axis == 1 ? n : (long)n * n;
#pragma omp parallel
        {
            cplx *line = malloc(sizeof(cplx) * n), *res = malloc(sizeof(cplx) * n);
#pragma omp for schedule(static)
            for (long l = 0; l < (long)n * n; ++l) {
                int u = (int)(l % n), v = (int)(l / n);
                long base = axis == 0 ? idx3(n, v, u, 0)
                          : axis == 1 ? idx3(n, v, 0, u)
                                      : idx3(n, 0, v, u);
                for (int i = 0; i < n; ++i) line[i] = a[base + i * st];
                fft_rec(n, line, 1, res, sign);
                for (int i = 0; i < n; ++i) a[base + i * st] = res[i];
            }
            free(line);
            free(res);
        }
    }
}

/* ------------------------------------------------------------------ */
/* Direct translational cross-correlation, Eqs. 1 and 3 as a Riemann    */
/* sum over the periodic grid:                                          */
/*   E[j] = h^3 sum_n rho1[n] rho2R[(n - j) mod N]                       */
/* O(N^6); only for small grids.                                        */
/* ------------------------------------------------------------------ */
void or_correlate_direct(int n, const double *rho1, const double *rho2r, double *E)
{
    const double h = 2.0 / n, dv = h * h * h;
#pragma omp parallel for schedule(dynamic)
    for (int jz = 0; jz < n; ++jz)
        for (int jy = 0; jy < n; ++jy)
            for (int jx = 0; jx < n; ++jx) {
                double acc = 0.0;
                for (int z = 0; z < n; ++z)
                    for (int y = 0; y < n; ++y)
                        for (int x = 0; x < n; ++x)
                            acc += rho1[idx3(n, z, y, x)] *
                                   rho2r[idx3(n, wrap(z - jz, n), wrap(y - jy, n), wrap(x - jx, n))];
                E[idx3(n, jz, jy, jx)] = dv * acc;
            }
}

/* signed frequency index in [-N/2, N/2) */
static int signed_k(int k, int n) { return k < (n + 1) / 2 ? k : k - n; }

/* ------------------------------------------------------------------ */
/* Energy and force over all lags through the convolution theorem,      */
/* Eqs. 5 and 6a (Section 2.4) discretised per Section 3.2:             */
/*   S_k   = h^3 * rho1^_k * conj(rho2R^_k)     (reflection = conj for   */
/*                                               real densities)         */
/*   E     = IDFT(S) / N^3                                               */
/*   F_d   = -IDFT(2 pi i omega_d S) / N^3,  omega_d = k~_d / (N h),     */
/*           multiplier 0 on each axis' Nyquist index (even N).          */
/* Outputs are real parts; E and F are real for real densities.         */
/* ------------------------------------------------------------------ */
void or_fields_spec(int n, const double *rho1, const double *b_ri,
                    double *E, double *Fx, double *Fy, double *Fz);

void or_fields(int n, const double *rho1, const double *rho2r,
               double *E, double *Fx, double *Fy, double *Fz)
{
    const long m = (long)n * n * n;
    cplx *B = malloc(sizeof(cplx) * m);
    for (long i = 0; i < m; ++i) B[i] = rho2r[i];
    or_fft3d(n, (double *)B, -1);
    or_fields_spec(n, rho1, (const double *)B, E, Fx, Fy, Fz);
    free(B);
}

/* The same fields given the moving density's (rotated) spectrum B = DFT(rho2R)
 * directly, natural order, complex interleaved. */
void or_fields_spec(int n, const double *rho1, const double *b_ri,
                    double *E, double *Fx, double *Fy, double *Fz)
{
    const long m = (long)n * n * n;
    const double h = 2.0 / n, dv = h * h * h;
    const cplx *B = (const cplx *)b_ri;
    cplx *A = malloc(sizeof(cplx) * m);
    cplx *S = malloc(sizeof(cplx) * m), *G = malloc(sizeof(cplx) * m);
    for (long i = 0; i < m; ++i) A[i] = rho1[i];
    or_fft3d(n, (double *)A, -1);
    for (long i = 0; i < m; ++i) S[i] = dv * A[i] * conj(B[i]);

    memcpy(G, S, sizeof(cplx) * m);
    or_fft3d(n, (double *)G, +1);
    for (long i = 0; i < m; ++i) E[i] = creal(G[i]) / (double)m;

    double *outs[3] = {Fx, Fy, Fz};
    for (int d = 0; d < 3; ++d) {
        for (int kz = 0; kz < n; ++kz)
            for (int ky = 0; ky < n; ++ky)
                for (int kx = 0; kx < n; ++kx) {
                    int kd = d == 0 ? kx : d == 1 ? ky : kz;
                    double kt = (n % 2 == 0 && kd == n / 2) ? 0.0 : (double)signed_k(kd, n);
                    double omega = kt / (n * h);
                    long i = idx3(n, kz, ky, kx);
                    G[i] = 2.0 * PI * I * omega * S[i];
                }
        or_fft3d(n, (double *)G, +1);
        for (long i = 0; i < m; ++i) outs[d][i] = -creal(G[i]) / (double)m;
    }
    free(A); free(S); free(G);
}

/* ------------------------------------------------------------------ */
/* Mesh descriptor, Eq. 2 (Section 2.3, "Skeletal Density"; Section 3.1), */
/* for a closed triangle mesh with outward orientation:                   */
/*   PMC   winding number W(p) = (1/4 pi) sum of the triangles' signed     */
/*         solid angles (Eq. 2 with the inverse-square kernel), W = 1      */
/*         inside, 0 outside;                                              */
/*   xi    signed distance, -min_q |p - q| inside, + outside;              */
/*   rho   (1/4 pi) integral over the surface of g(eta/|xi| - 1) d gamma,  */
/*         g(x) = exp(-x^2 / 2 sigma^2), eta = |p - q|, d gamma the signed */
/*         solid-angle element (= eta^-2 dA_perp): the inverse-square      */
/*         kernel times the Gaussian that weights approximate nearest      */
/*         boundary points, so rho -> W as sigma -> infinity.              */
/* The integral is a Riemann sum over triangles subdivided (4 ways, at the */
/* edge midpoints) until each piece subtends at most gamma_max or depth    */
/* dmax is reached; a piece contributes g at its centroid times its exact  */
/* solid angle (solid angles add up, so subdividing never changes the      */
/* g = 1 limit).                                                           */
/* ------------------------------------------------------------------ */
static void sub3(const double *a, const double *b, double *o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/* signed solid angle of triangle (A, B, C) seen from p (van Oosterom and
 * Strackee's formula): positive when p is on the side opposite the normal
 * (B - A) x (C - A) */
static double solid_angle(const double *p, const double *A, const double *B, const double *C)
{
    double a[3], b[3], c[3], bc[3];
    sub3(A, p, a); sub3(B, p, b); sub3(C, p, c);
    cross3(b, c, bc);
    const double la = sqrt(dot3(a, a)), lb = sqrt(dot3(b, b)), lc = sqrt(dot3(c, c));
    const double num = dot3(a, bc);
    const double den = la * lb * lc + dot3(a, b) * lc + dot3(a, c) * lb + dot3(b, c) * la;
    return 2.0 * atan2(num, den);
}

/* distance from p to triangle (A, B, C): the closest point lies in the face,
 * on an edge or at a vertex; the face case by barycentric coordinates of
 * the projection, the others by clamped projections onto the edges */
static double tri_distance(const double *p, const double *A, const double *B, const double *C)
{
    double e0[3], e1[3], v[3], nrm[3];
    sub3(B, A, e0); sub3(C, A, e1); sub3(p, A, v);
    cross3(e0, e1, nrm);
    const double a00 = dot3(e0, e0), a01 = dot3(e0, e1), a11 = dot3(e1, e1);
    const double b0 = dot3(v, e0), b1 = dot3(v, e1);
    const double det = a00 * a11 - a01 * a01;
    if (det > 0) {
        const double s = (a11 * b0 - a01 * b1) / det, t = (a00 * b1 - a01 * b0) / det;
        if (s >= 0 && t >= 0 && s + t <= 1) {
            const double nn = sqrt(dot3(nrm, nrm));
            return fabs(dot3(v, nrm)) / nn;
        }
    }
    const double *P[3] = {A, B, C};
    double best = INFINITY;
    for (int k = 0; k < 3; ++k) {
        const double *X = P[k], *Y = P[(k + 1) % 3];
        double e[3], w[3];
        sub3(Y, X, e); sub3(p, X, w);
        double t = dot3(w, e) / dot3(e, e);
        t = t < 0 ? 0 : t > 1 ? 1 : t;
        const double d[3] = {w[0] - t * e[0], w[1] - t * e[1], w[2] - t * e[2]};
        const double dd = sqrt(dot3(d, d));
        if (dd < best) best = dd;
    }
    return best;
}

static double mesh_sdf_piece(const double *p, const double *A, const double *B, const double *C, double axi,
                             double sigma, double gamma_max, int depth, int dmax)
{
    const double om = solid_angle(p, A, B, C);
    if (fabs(om) > gamma_max && depth < dmax) {
        double ab[3], bc[3], ca[3];
        for (int i = 0; i < 3; ++i) {
            ab[i] = 0.5 * (A[i] + B[i]);
            bc[i] = 0.5 * (B[i] + C[i]);
            ca[i] = 0.5 * (C[i] + A[i]);
        }
        return mesh_sdf_piece(p, A, ab, ca, axi, sigma, gamma_max, depth + 1, dmax) +
               mesh_sdf_piece(p, ab, B, bc, axi, sigma, gamma_max, depth + 1, dmax) +
               mesh_sdf_piece(p, ca, bc, C, axi, sigma, gamma_max, depth + 1, dmax) +
               mesh_sdf_piece(p, ab, bc, ca, axi, sigma, gamma_max, depth + 1, dmax);
    }
    const double q[3] = {(A[0] + B[0] + C[0]) / 3, (A[1] + B[1] + C[1]) / 3, (A[2] + B[2] + C[2]) / 3};
    double d[3];
    sub3(q, p, d);
    const double eta = sqrt(dot3(d, d));
    const double x = eta / axi - 1.0;
    return exp(-0.5 * x * x / (sigma * sigma)) * om;
}

/* On the N^3 nodes: W (winding number), XI (signed distance), RHO (descriptor). */
void or_mesh_sdf(int n, int nv, const double *V, int nt, const int *T, double sigma, double gamma_max, int dmax,
                 double *W, double *XI, double *RHO)
{
    const double h = 2.0 / n;
    (void)nv;
#pragma omp parallel for schedule(dynamic)
    for (long i = 0; i < (long)n * n * n; ++i) {
        const int x = (int)(i % n), y = (int)((i / n) % n), z = (int)(i / ((long)n * n));
        const double p[3] = {-1.0 + x * h, -1.0 + y * h, -1.0 + z * h};
        double w = 0, dist = INFINITY;
        for (int t = 0; t < nt; ++t) {
            const double *A = V + 3 * T[3 * t], *B = V + 3 * T[3 * t + 1], *C = V + 3 * T[3 * t + 2];
            w += solid_angle(p, A, B, C);
            const double d = tri_distance(p, A, B, C);
            if (d < dist) dist = d;
        }
        w /= 4.0 * PI;
        const double xi = w >= 0.5 ? -dist : dist;
        double rho = 0;
        if (dist > 1e-12)
            for (int t = 0; t < nt; ++t)
                rho += mesh_sdf_piece(p, V + 3 * T[3 * t], V + 3 * T[3 * t + 1], V + 3 * T[3 * t + 2], dist, sigma,
                                      gamma_max, 0, dmax);
        W[i] = w;
        XI[i] = xi;
        RHO[i] = rho / (4.0 * PI);
    }
}

/* ------------------------------------------------------------------ */
/* Analytic torque field, the rotational gradient of Eq. 6b.  For world-  */
/* frame perturbations R -> exp(theta [e_a]x) R of the moving part about  */
/* its reference point (at t),                                           */
/*   T_a(t) = -dE/dtheta_a = integral rho1(t + r) (r x grad rho2R(r))_a dr */
/* (Eq. 6b's moment field r rho2).  Integrating by parts moves the moment */
/* onto the stationary part:                                             */
/*   T(t) = C(G, rho2R)(t) - t x F(t),  G(u) = -u x grad rho1(u),         */
/* with C the correlation that gives E (Eqs. 3, 5) and F the force.      */
/* Discretisation: grad rho1 is the spectral derivative (multiplier      */
/* 2 pi i omega, Nyquist 0, as for the force), u_n = -1 + n h per axis,   */
/* t the signed lag j~ h; outputs the three torque fields.                */
/* ------------------------------------------------------------------ */
void or_torque_analytic(int n, const double *rho1, const double *rho2r, double *Tx, double *Ty, double *Tz)
{
    const long m = (long)n * n * n;
    const double h = 2.0 / n, dv = h * h * h;
    cplx *A = malloc(sizeof(cplx) * m), *B = malloc(sizeof(cplx) * m), *W = malloc(sizeof(cplx) * m);
    double *g[3], *F[3];
    for (int d = 0; d < 3; ++d) { g[d] = malloc(sizeof(double) * m); F[d] = malloc(sizeof(double) * m); }
    for (long i = 0; i < m; ++i) { A[i] = rho1[i]; B[i] = rho2r[i]; }
    or_fft3d(n, (double *)A, -1);
    or_fft3d(n, (double *)B, -1);
    /* grad rho1, spectrally */
    for (int d = 0; d < 3; ++d) {
        for (int kz = 0; kz < n; ++kz)
            for (int ky = 0; ky < n; ++ky)
                for (int kx = 0; kx < n; ++kx) {
                    const int kd = d == 0 ? kx : d == 1 ? ky : kz;
                    const double kt = (n % 2 == 0 && kd == n / 2) ? 0.0 : (double)signed_k(kd, n);
                    const long i = idx3(n, kz, ky, kx);
                    W[i] = 2.0 * PI * I * (kt / (n * h)) * A[i];
                }
        or_fft3d(n, (double *)W, +1);
        for (long i = 0; i < m; ++i) g[d][i] = creal(W[i]) / (double)m;
    }
    /* force field of the pair (for the t x F term) */
    double *E = malloc(sizeof(double) * m);
    or_fields(n, rho1, rho2r, E, F[0], F[1], F[2]);
    free(E);
    double *outs[3] = {Tx, Ty, Tz};
    for (int a = 0; a < 3; ++a) {
        /* G_a = -(u x grad rho1)_a */
        for (int z = 0; z < n; ++z)
            for (int y = 0; y < n; ++y)
                for (int x = 0; x < n; ++x) {
                    const double u[3] = {-1.0 + x * h, -1.0 + y * h, -1.0 + z * h};
                    const long i = idx3(n, z, y, x);
                    const double gx = g[0][i], gy = g[1][i], gz = g[2][i];
                    const double c = a == 0 ? u[1] * gz - u[2] * gy : a == 1 ? u[2] * gx - u[0] * gz : u[0] * gy - u[1] * gx;
                    W[i] = -c;
                }
        or_fft3d(n, (double *)W, -1);
        for (long i = 0; i < m; ++i) W[i] = dv * W[i] * conj(B[i]);
        or_fft3d(n, (double *)W, +1);
        for (int jz = 0; jz < n; ++jz)
            for (int jy = 0; jy < n; ++jy)
                for (int jx = 0; jx < n; ++jx) {
                    const long i = idx3(n, jz, jy, jx);
                    const double t[3] = {signed_k(jx, n) * h, signed_k(jy, n) * h, signed_k(jz, n) * h};
                    const double f[3] = {F[0][i], F[1][i], F[2][i]};
                    const double txf = a == 0 ? t[1] * f[2] - t[2] * f[1] : a == 1 ? t[2] * f[0] - t[0] * f[2] : t[0] * f[1] - t[1] * f[0];
                    outs[a][i] = creal(W[i]) / (double)m - txf;
                }
    }
    for (int d = 0; d < 3; ++d) { free(g[d]); free(F[d]); }
    free(A); free(B); free(W);
}

/* ------------------------------------------------------------------ */
/* Rotation in the frequency domain, Section 3.2 step 1: the spectrum   */
/* of the rotated density rho2(R^T p) is rho2^(R^T omega), read off a   */
/* precomputed spectrum by trilinear interpolation.                     */
/*                                                                      */
/* Table: rho2 zero-padded to N' = os N nodes per axis (same spacing h, */
/* box [-os, os)^3, the original nodes at the centre) and transformed;  */
/* the phase is taken about the physical origin rather than the box     */
/* corner: table[k'] = (-1)^(kx'+ky'+kz') DFT_N'(pad rho2)[k'], so a     */
/* density centred at the origin has a smooth table.  Frequency k' of   */
/* the table is omega = k'/(2 os); frequency k of the N grid is         */
/* omega = k/2, index os*k in the table.                                */
/* ------------------------------------------------------------------ */
void or_spectral_table(int n, int os, const double *rho, double *table_ri)
{
    const int np = os * n, off = (np - n) / 2;
    const long mp = (long)np * np * np;
    cplx *T = (cplx *)table_ri;
    for (long i = 0; i < mp; ++i) T[i] = 0.0;
    for (int z = 0; z < n; ++z)
        for (int y = 0; y < n; ++y)
            for (int x = 0; x < n; ++x)
                T[idx3(np, z + off, y + off, x + off)] = rho[idx3(n, z, y, x)];
    or_fft3d(np, table_ri, -1);
    for (int kz = 0; kz < np; ++kz)
        for (int ky = 0; ky < np; ++ky)
            for (int kx = 0; kx < np; ++kx)
                if ((kx + ky + kz) & 1) T[idx3(np, kz, ky, kx)] = -T[idx3(np, kz, ky, kx)];
}

/* Periodic trilinear interpolation of a complex n^3 table at index u. */
static cplx trilinear_c(int n, const cplx *g, const double u[3])
{
    long i0[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        const double fl = floor(u[a]);
        i0[a] = (long)fl;
        f[a] = u[a] - fl;
    }
    cplx acc = 0.0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                const double w = (dx ? f[0] : 1 - f[0]) * (dy ? f[1] : 1 - f[1]) * (dz ? f[2] : 1 - f[2]);
                acc += w * g[idx3(n, wrap(i0[2] + dz, n), wrap(i0[1] + dy, n), wrap(i0[0] + dx, n))];
            }
    return acc;
}

/* Rotated spectrum on the N grid (natural order): for every frequency k   */
/* with signed index k~, B[k] = (-1)^(kx+ky+kz) trilinear(table, os R^T k~), */
/* and B = 0 wherever an axis index is the Nyquist index N/2 (a rotated     */
/* frequency has no Nyquist partner, so those planes are left out).         */
void or_spectral_rotate(int n, int os, const double *table_ri, const double *R, double *out_ri)
{
    const int np = os * n;
    const cplx *T = (const cplx *)table_ri;
    cplx *B = (cplx *)out_ri;
#pragma omp parallel for schedule(static)
    for (int kz = 0; kz < n; ++kz)
        for (int ky = 0; ky < n; ++ky)
            for (int kx = 0; kx < n; ++kx) {
                const long i = idx3(n, kz, ky, kx);
                if (2 * kx == n || 2 * ky == n || 2 * kz == n) { B[i] = 0.0; continue; }
                const double k[3] = {signed_k(kx, n), signed_k(ky, n), signed_k(kz, n)};
                double u[3];
                for (int a = 0; a < 3; ++a)  /* (R^T k)_a = sum_b R[b][a] k_b */
                    u[a] = os * (R[0 * 3 + a] * k[0] + R[1 * 3 + a] * k[1] + R[2 * 3 + a] * k[2]);
                const cplx v = trilinear_c(np, T, u);
                B[i] = ((kx + ky + kz) & 1) ? -v : v;
            }
}

/* Periodic trilinear interpolation of a complex table and its gradient
 * (d/du_x, d/du_y, d/du_z in index units) at u. */
static cplx trilinear_c_grad(int n, const cplx *g, const double u[3], cplx grad[3])
{
    long i0[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        const double fl = floor(u[a]);
        i0[a] = (long)fl;
        f[a] = u[a] - fl;
    }
    cplx c[2][2][2];
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx)
                c[dz][dy][dx] = g[idx3(n, wrap(i0[2] + dz, n), wrap(i0[1] + dy, n), wrap(i0[0] + dx, n))];
    cplx v = 0.0;
    grad[0] = grad[1] = grad[2] = 0.0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                const double wx = dx ? f[0] : 1 - f[0], wy = dy ? f[1] : 1 - f[1], wz = dz ? f[2] : 1 - f[2];
                const double sx = dx ? 1 : -1, sy = dy ? 1 : -1, sz = dz ? 1 : -1;
                v += wx * wy * wz * c[dz][dy][dx];
                grad[0] += sx * wy * wz * c[dz][dy][dx];
                grad[1] += wx * sy * wz * c[dz][dy][dx];
                grad[2] += wx * wy * sz * c[dz][dy][dx];
            }
    return v;
}

/* ------------------------------------------------------------------ */
/* Single-pose evaluation with truncated spectra, Section 4.2            */
/* ("Truncated Inverse FFT") with the low-pass filtering of Section 3.3: */
/* only the modes with |k~_a| <= K on every axis are kept, and the       */
/* inverse transform is summed at the one translation t instead of over  */
/* the grid:                                                             */
/*   S(k)  = (h^3/N^3) rho1^(k) conj(B(k)),  B(k) = (-1)^(kx+ky+kz)       */
/*           trilinear(table, os R^T k~)   (Section 3.2, step 1)          */
/*   E     = sum_k Re S(k) exp(i pi k~.t)    (omega = k~/2, N h = 2)      */
/*   F_d   = -sum_k Re i pi k~_d S(k) exp(i pi k~.t)        (Eq. 6a)      */
/*   T_a   = -dE/dtheta_a for R -> exp(theta [e_a]x) R: the exact         */
/*           derivative of the interpolated model, d(os R^T k~)/dtheta_a  */
/*           = -os R^T (e_a x k~)                                         */
/* out7 = (E, Fx, Fy, Fz, Tx, Ty, Tz).                                    */
/* ------------------------------------------------------------------ */
void or_lowpass(int n, const double *rho1, const double *table_ri, int os, int K, const double *R,
                const double *t, double *out7)
{
    const long m = (long)n * n * n;
    const int np = os * n;
    const double h = 2.0 / n, scale = h * h * h / (double)m;
    const cplx *T = (const cplx *)table_ri;
    cplx *A = malloc(sizeof(cplx) * m);
    for (long i = 0; i < m; ++i) A[i] = rho1[i];
    or_fft3d(n, (double *)A, -1);
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int kz = -K; kz <= K; ++kz)
        for (int ky = -K; ky <= K; ++ky)
            for (int kx = -K; kx <= K; ++kx) {
                const double k[3] = {kx, ky, kz};
                double u[3];
                for (int a = 0; a < 3; ++a)
                    u[a] = os * (R[0 * 3 + a] * k[0] + R[1 * 3 + a] * k[1] + R[2 * 3 + a] * k[2]);
                cplx grad[3];
                cplx b = trilinear_c_grad(np, T, u, grad);
                const int odd = (kx + ky + kz) & 1;
                if (odd) { b = -b; grad[0] = -grad[0]; grad[1] = -grad[1]; grad[2] = -grad[2]; }
                const cplx a1 = scale * A[idx3(n, wrap(kz, n), wrap(ky, n), wrap(kx, n))];
                const cplx ph = cexp(I * PI * (k[0] * t[0] + k[1] * t[1] + k[2] * t[2]));
                const cplx term = a1 * conj(b) * ph;
                acc[0] += creal(term);
                for (int d = 0; d < 3; ++d) acc[1 + d] -= creal(I * PI * k[d] * term);
                for (int ax = 0; ax < 3; ++ax) {
                    /* v = -os R^T (e_a x k) */
                    double ek[3] = {0, 0, 0};
                    if (ax == 0) { ek[1] = -k[2]; ek[2] = k[1]; }
                    else if (ax == 1) { ek[0] = k[2]; ek[2] = -k[0]; }
                    else { ek[0] = -k[1]; ek[1] = k[0]; }
                    cplx db = 0.0;
                    for (int c = 0; c < 3; ++c) {
                        const double vc = -os * (R[0 * 3 + c] * ek[0] + R[1 * 3 + c] * ek[1] + R[2 * 3 + c] * ek[2]);
                        db += grad[c] * vc;
                    }
                    acc[4 + ax] -= creal(a1 * conj(db) * ph);
                }
            }
    for (int i = 0; i < 7; ++i) out7[i] = acc[i];
    free(A);
}

/* Geodesic angle between two unit quaternions (double cover aware). */
static double quat_angle(const double *a, const double *b)
{
    double d = fabs(a[0] * b[0] + a[1] * b[1] + a[2] * b[2] + a[3] * b[3]);
    if (d > 1.0) d = 1.0;
    return 2.0 * acos(d);
}

/* indices of the k smallest angles (ties to the lower index), excluding `skip` */
static void k_nearest(int nrot, const double *quats, const double *q, int skip,
                      int k, int *out_idx, double *out_ang)
{
    for (int s = 0; s < k; ++s) { out_idx[s] = -1; out_ang[s] = INFINITY; }
    for (int j = 0; j < nrot; ++j) {
        if (j == skip) continue;
        double th = quat_angle(q, quats + 4 * j);
        /* insertion into the sorted k-list; strict '<' keeps lower index on ties */
        int pos = k;
        while (pos > 0 && th < out_ang[pos - 1]) --pos;
        if (pos < k) {
            for (int s = k - 1; s > pos; --s) { out_ang[s] = out_ang[s - 1]; out_idx[s] = out_idx[s - 1]; }
            out_ang[pos] = th;
            out_idx[pos] = j;
        }
    }
}

/* Matrix logarithm on SO(3): the axis-angle vector of M. */
static void so3_log(const double *M, double *v)
{
    double c = (M[0] + M[4] + M[8] - 1.0) / 2.0;
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    double th = acos(c);
    double w[3] = {M[7] - M[5], M[2] - M[6], M[3] - M[1]}; /* 2 sin(th) * axis */
    if (th < 1e-6) { /* th/(2 sin th) -> 1/2 */
        for (int a = 0; a < 3; ++a) v[a] = 0.5 * w[a];
        return;
    }
    if (PI - th < 1e-6) { /* axis from the symmetric part: M + I = 2 a a^T */
        int best = 0;
        for (int a = 1; a < 3; ++a) if (M[4 * a] > M[4 * best]) best = a;
        double ax[3];
        double d = sqrt((M[4 * best] + 1.0) / 2.0);
        for (int a = 0; a < 3; ++a) ax[a] = (a == best) ? d : (M[3 * a + best] + M[3 * best + a]) / (4.0 * d);
        for (int a = 0; a < 3; ++a) v[a] = th * ax[a];
        return;
    }
    double s = th / (2.0 * sin(th));
    for (int a = 0; a < 3; ++a) v[a] = s * w[a];
}

/* ------------------------------------------------------------------ */
/* Torque field by least-squares finite differences across rotations.   */
/* The paper's rotational gradient is Eq. 6b; this path estimates the   */
/* same quantity, T = -dE/d(theta) for world-frame perturbations        */
/* R_j = exp([theta]x) R_i, from the energy fields of the k nearest     */
/* sampled rotations:                                                   */
/*   A (k x 3) rows = Log(R_j R_i^T),  b_j = E_j - E_i per cell,        */
/*   g = (A^T A)^{-1} A^T b,  T = -g.                                   */
/* E is nrot consecutive n^3 fields; T is nrot x 3 consecutive fields. */
/* status[i] = 0 on success, 1 when A^T A is singular (cond > 1e16),   */
/* in which case rotation i's torque is NaN.                            */
/* ------------------------------------------------------------------ */
void or_torque(int n, int nrot, const double *quats, const double *E, int knn,
               double *T, int *status)
{
    const long m = (long)n * n * n;
    for (int i = 0; i < nrot; ++i) {
        int *nb = malloc(sizeof(int) * knn);
        double *ang = malloc(sizeof(double) * knn);
        double *A = malloc(sizeof(double) * 3 * knn);
        k_nearest(nrot, quats, quats + 4 * i, i, knn, nb, ang);
        double Ri[9], Rj[9], M[9];
        or_quat_to_rot(quats + 4 * i, Ri);
        int ok = 1;
        for (int s = 0; s < knn; ++s) {
            if (nb[s] < 0) { ok = 0; break; }
            or_quat_to_rot(quats + 4 * nb[s], Rj);
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c)
                    M[3 * r + c] = Rj[3 * r + 0] * Ri[3 * c + 0] + Rj[3 * r + 1] * Ri[3 * c + 1] +
                                   Rj[3 * r + 2] * Ri[3 * c + 2];
            so3_log(M, A + 3 * s);
        }
        /* normal matrix and its inverse by the adjugate */
        double N3[9] = {0}, Ninv[9];
        for (int s = 0; s < knn && ok; ++s)
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) N3[3 * r + c] += A[3 * s + r] * A[3 * s + c];
        double det = N3[0] * (N3[4] * N3[8] - N3[5] * N3[7]) - N3[1] * (N3[3] * N3[8] - N3[5] * N3[6]) +
                     N3[2] * (N3[3] * N3[7] - N3[4] * N3[6]);
        double fro = 0;
        for (int e = 0; e < 9; ++e) fro += N3[e] * N3[e];
        if (ok) {
            Ninv[0] = (N3[4] * N3[8] - N3[5] * N3[7]) / det;
            Ninv[1] = (N3[2] * N3[7] - N3[1] * N3[8]) / det;
            Ninv[2] = (N3[1] * N3[5] - N3[2] * N3[4]) / det;
            Ninv[3] = (N3[5] * N3[6] - N3[3] * N3[8]) / det;
            Ninv[4] = (N3[0] * N3[8] - N3[2] * N3[6]) / det;
            Ninv[5] = (N3[2] * N3[3] - N3[0] * N3[5]) / det;
            Ninv[6] = (N3[3] * N3[7] - N3[4] * N3[6]) / det;
            Ninv[7] = (N3[1] * N3[6] - N3[0] * N3[7]) / det;
            Ninv[8] = (N3[0] * N3[4] - N3[1] * N3[3]) / det;
            double finv = 0;
            for (int e = 0; e < 9; ++e) finv += Ninv[e] * Ninv[e];
            /* Frobenius condition number of the normal matrix */
            if (!(det != 0.0) || !isfinite(finv) || sqrt(fro) * sqrt(finv) > 1e16) ok = 0;
        }
        status[i] = ok ? 0 : 1;
        double *Ti = T + (long)i * 3 * m;
        if (!ok) {
            for (long c = 0; c < 3 * m; ++c) Ti[c] = NAN;
        } else {
            /* P = (A^T A)^{-1} A^T, 3 x k */
            double *P = malloc(sizeof(double) * 3 * knn);
            for (int r = 0; r < 3; ++r)
                for (int s = 0; s < knn; ++s)
                    P[r * knn + s] = Ninv[3 * r + 0] * A[3 * s + 0] + Ninv[3 * r + 1] * A[3 * s + 1] +
                                     Ninv[3 * r + 2] * A[3 * s + 2];
            const double *Ei = E + (long)i * m;
#pragma omp parallel for schedule(static)
            for (long c = 0; c < m; ++c) {
                double g[3] = {0, 0, 0};
                for (int s = 0; s < knn; ++s) {
                    double b = E[(long)nb[s] * m + c] - Ei[c];
                    for (int r = 0; r < 3; ++r) g[r] += P[r * knn + s] * b;
                }
                for (int r = 0; r < 3; ++r) Ti[r * m + c] = -g[r];
            }
            free(P);
        }
        free(nb); free(ang); free(A);
    }
}

/* ------------------------------------------------------------------ */
/* Pose query for the restricted-orientation mode (Section 4.2,         */
/* "Restricted Motion DOF"): fields precomputed per sampled rotation    */
/* are read at an arbitrary pose (t, q).                                */
/*   rotation: the k sampled rotations nearest to q (geodesic angle),   */
/*             weights proportional to 1/theta_j and normalised; an     */
/*             exact hit (theta < 1e-12) returns that rotation alone.   */
/*   translation: periodic trilinear interpolation over the lag grid at */
/*             u = t/h (lag index j <-> translation j*h).               */
/* fields: nrot x nf consecutive n^3 arrays; out: nf values.            */
/* ------------------------------------------------------------------ */
void or_query(int n, int nrot, const double *quats, const double *fields, int nf,
              const double *t, const double *q, int k, double *out)
{
    const long m = (long)n * n * n;
    const double h = 2.0 / n;
    int *nb = malloc(sizeof(int) * k);
    double *ang = malloc(sizeof(double) * k), *w = malloc(sizeof(double) * k);
    double qn[4];
    double nrm = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int a = 0; a < 4; ++a) qn[a] = q[a] / nrm;
    k_nearest(nrot, quats, qn, -1, k, nb, ang);
    int used = k;
    if (ang[0] < 1e-12) {
        used = 1;
        w[0] = 1.0;
    } else {
        double sw = 0;
        for (int s = 0; s < k; ++s) { w[s] = 1.0 / ang[s]; sw += w[s]; }
        for (int s = 0; s < k; ++s) w[s] /= sw;
    }
    double u[3] = {t[0] / h, t[1] / h, t[2] / h};
    for (int f = 0; f < nf; ++f) {
        double acc = 0;
        for (int s = 0; s < used; ++s)
            acc += w[s] * trilinear(n, fields + ((long)nb[s] * nf + f) * m, u);
        out[f] = acc;
    }
    free(nb); free(ang); free(w);
}

/* k nearest sampled rotations to q (exposed for tests). */
void or_nearest(int nrot, const double *quats, const double *q, int skip, int k,
                int *idx, double *ang)
{
    k_nearest(nrot, quats, q, skip, k, idx, ang);
}

void or_so3_log(const double *M, double *v) { so3_log(M, v); }
