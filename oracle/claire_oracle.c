/*
 * claire_oracle.c -- plain, slow, FP64 CPU oracle for the Gauss-Newton-Krylov
 * diffeomorphic registration method of Brunn, Himthani, Biros, Mehl and Mang,
 * "Multi-Node Multi-GPU Diffeomorphic Image Registration for Large-Scale
 * Imaging Problems" (arXiv 2008.12820).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker for the CUDA path: only
 * the tests, the smoke check and the benchmark's CPU-baseline leg may build,
 * load or call it.  It shares no code, header, table or helper with the CUDA
 * library, and the library never calls it (there is no CPU fallback).
 *
 * Everything here is written for a reader who checks it against the paper by
 * eye: no blocking, no fusion, no reordering beyond what each definition states.
 * Floating point is IEEE double throughout.
 *
 * Conventions (paper, Section 3 "Discretization"):
 *   domain Omega = [0, 2*pi)^3, periodic; grid x_ijk = (i*h1, j*h2, k*h3),
 *   h_d = 2*pi/N_d; x3 is the contiguous axis (Section 4.3), so
 *   idx(i1,i2,i3) = (i1*N2 + i2)*N3 + i3.  Vector fields are three scalar
 *   fields one after another (component-major).  Time step dt = 1/N_t.
 *
 * Readings of points the paper leaves open (each is also listed in the design
 * notes of the repository):
 *   - regularization: beta*A := -beta*Laplace - gamma*grad(div), i.e. the H1
 *     seminorm plus a divergence penalty (Section 2.1, Eq. (3.1));
 *   - zero wavenumber of (beta*A)^{-1}: identity;
 *   - Nyquist index of an even axis: its first-derivative wavenumber is 0,
 *     |k|^2 keeps (N/2)^2;
 *   - RK2 for the characteristics is Heun's method, v at the predictor point
 *     by cubic interpolation;
 *   - source terms along characteristics (adjoint lambda*div v, incremental
 *     state -vt.grad m) by the trapezoidal (Heun) rule along the characteristic;
 *   - the time integral of the body force by the trapezoidal rule;
 *   - L2 inner products are h1*h2*h3-weighted sums.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double _Complex cplx;

#define OR_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------------- */
/* Grid helpers                                                               */
/* ------------------------------------------------------------------------- */

static inline long or_idx(const int n[3], long i1, long i2, long i3) {
    return (i1 * n[1] + i2) * n[2] + i3;
}

/* periodic wrap of an integer index into [0, n) */
static inline long or_wrap(long i, long n) {
    long r = i % n;
    return r < 0 ? r + n : r;
}

/* integer wavenumber of FFT index i on an axis of n points: 0..ceil(n/2)-1
 * map to themselves, the rest to i-n; for even n the Nyquist index n/2 maps to
 * -n/2 (only its square is ever used). */
static inline double or_wavenumber(int i, int n) {
    return (2 * i < n) ? (double)i : (double)(i - n);
}

/* wavenumber used for first derivatives: as above, but 0 at the Nyquist index
 * of an even axis (the sine mode at Nyquist vanishes on the grid). */
static inline double or_wavenumber_d1(int i, int n) {
    if ((n % 2 == 0) && (2 * i == n)) return 0.0;
    return or_wavenumber(i, n);
}

/* ------------------------------------------------------------------------- */
/* 1D DFT by recursive mixed-radix Cooley-Tukey (decimation in time)          */
/*   out[k] = sum_j in[j*stride] * exp(sign * 2*pi*i * j*k / n)               */
/* Every prime factor p of n is handled by a direct p-point sum.               */
/* ------------------------------------------------------------------------- */

static int or_smallest_factor(int n) {
    for (int p = 2; p * p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

/* roots of unity exp(sign*2*pi*i*t/n), t = 0..n-1, each from cos/sin of the
 * exact angle */
static cplx *or_roots(int n, int sign) {
    cplx *w = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    for (int t = 0; t < n; ++t) {
        double a = 2.0 * OR_PI * (double)t / (double)n;
        w[t] = cos(a) + (double)sign * sin(a) * I;
    }
    return w;
}

/* w holds the n0-th roots of unity; a sub-transform of length n uses
 * w_n^t = w[(t mod n) * (n0 / n)] */
static void or_dft_rec(const cplx *in, long stride, cplx *out, int n, const cplx *w, int n0) {
    if (n == 1) { out[0] = in[0]; return; }
    int p = or_smallest_factor(n);
    int m = n / p;
    long step = n0 / n;
    /* p sub-transforms of length m over the residues r mod p:
     * Y_r[k] = sum_j in[(p*j + r)*stride] w_m^{jk}, stored at out[r*m + k]. */
    for (int r = 0; r < p; ++r)
        or_dft_rec(in + (long)r * stride, stride * p, out + (long)r * m, m, w, n0);
    /* combine: X[k + q*m] = sum_r w_n^{r(k + q*m)} Y_r[k] */
    cplx ybuf[16];
    cplx *y = p <= 16 ? ybuf : (cplx *)malloc(sizeof(cplx) * (size_t)p);
    for (int k = 0; k < m; ++k) {
        for (int r = 0; r < p; ++r) y[r] = out[(long)r * m + k];
        for (int q = 0; q < p; ++q) {
            cplx s = 0;
            for (int r = 0; r < p; ++r)
                s += y[r] * w[(((long)r * (k + (long)q * m)) % n) * step];
            out[k + (long)q * m] = s;
        }
    }
    if (y != ybuf) free(y);
}

/* Unnormalized 3D DFT in place along all three axes; sign = -1 forward,
 * +1 backward.  Applied axis by axis as 1D transforms of every grid line. */
void or_fft3(int n1, int n2, int n3, double *data_ri, int sign) {
    const int n[3] = {n1, n2, n3};
    cplx *a = (cplx *)data_ri;
    for (int axis = 0; axis < 3; ++axis) {
        int len = n[axis];
        long stride = axis == 0 ? (long)n2 * n3 : (axis == 1 ? (long)n3 : 1);
        /* the lines of this axis: all index pairs of the other two axes */
        long nlines = ((long)n1 * n2 * n3) / len;
        cplx *w = or_roots(len, sign);
        #pragma omp parallel
        {
            cplx *line = (cplx *)malloc(sizeof(cplx) * (size_t)len);
            cplx *res = (cplx *)malloc(sizeof(cplx) * (size_t)len);
            #pragma omp for schedule(static)
            for (long l = 0; l < nlines; ++l) {
                long base;
                if (axis == 0) base = l;                                        /* (i2,i3) */
                else if (axis == 1) base = (l / n3) * (long)n2 * n3 + (l % n3); /* (i1,i3) */
                else base = l * n3;                                             /* (i1,i2) */
                for (int j = 0; j < len; ++j) line[j] = a[base + (long)j * stride];
                or_dft_rec(line, 1, res, len, w, len);
                for (int j = 0; j < len; ++j) a[base + (long)j * stride] = res[j];
            }
            free(line);
            free(res);
        }
        free(w);
    }
}

/* real field -> full complex spectrum (forward, unnormalized) */
static cplx *or_spectrum(const int n[3], const double *f) {
    long N = (long)n[0] * n[1] * n[2];
    cplx *F = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    for (long i = 0; i < N; ++i) F[i] = f[i];
    or_fft3(n[0], n[1], n[2], (double *)F, -1);
    return F;
}

/* complex spectrum -> real field: backward transform, divide by N, real part */
static void or_field(const int n[3], cplx *F, double *f) {
    long N = (long)n[0] * n[1] * n[2];
    or_fft3(n[0], n[1], n[2], (double *)F, +1);
    for (long i = 0; i < N; ++i) f[i] = creal(F[i]) / (double)N;
}

/* ------------------------------------------------------------------------- */
/* Spectral differential operators (Section 3 "Discretization")               */
/* ------------------------------------------------------------------------- */

/* gradient of a scalar field: d_d f = F^{-1}[ i*k_d * F f ] */
void or_grad(int n1, int n2, int n3, const double *f, double *g /* 3N */) {
    const int n[3] = {n1, n2, n3};
    long N = (long)n1 * n2 * n3;
    cplx *F = or_spectrum(n, f);
    cplx *G = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    for (int d = 0; d < 3; ++d) {
        #pragma omp parallel for collapse(2) schedule(static)
        for (int i1 = 0; i1 < n1; ++i1)
            for (int i2 = 0; i2 < n2; ++i2)
                for (int i3 = 0; i3 < n3; ++i3) {
                    const int ii[3] = {i1, i2, i3};
                    double kd = or_wavenumber_d1(ii[d], n[d]);
                    long id = or_idx(n, i1, i2, i3);
                    G[id] = I * kd * F[id];
                }
        or_field(n, G, g + d * N);
    }
    free(G);
    free(F);
}

/* divergence of a vector field: sum_d F^{-1}[ i*k_d * F v_d ] */
void or_div(int n1, int n2, int n3, const double *v /* 3N */, double *out) {
    const int n[3] = {n1, n2, n3};
    long N = (long)n1 * n2 * n3;
    cplx *S = (cplx *)calloc((size_t)N, sizeof(cplx));
    for (int d = 0; d < 3; ++d) {
        cplx *V = or_spectrum(n, v + d * N);
        #pragma omp parallel for collapse(2) schedule(static)
        for (int i1 = 0; i1 < n1; ++i1)
            for (int i2 = 0; i2 < n2; ++i2)
                for (int i3 = 0; i3 < n3; ++i3) {
                    const int ii[3] = {i1, i2, i3};
                    long id = or_idx(n, i1, i2, i3);
                    S[id] += I * or_wavenumber_d1(ii[d], n[d]) * V[id];
                }
        free(V);
    }
    or_field(n, S, out);
    free(S);
}

/* The 3x3 symbol of beta*A at wavenumber (k, khat):
 *   M = beta*|k|^2 * Id + gamma * khat khat^T
 * (vector Laplacian -beta*Laplace plus the divergence penalty -gamma*grad div). */
static void or_symbol_A(double beta, double gamma, const double k[3], const double kh[3],
                        double M[3][3]) {
    double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            M[a][b] = (a == b ? beta * k2 : 0.0) + gamma * kh[a] * kh[b];
}

/* Solve M x = r for a real 3x3 M and complex r by Gaussian elimination with
 * partial pivoting (real and imaginary parts share the same real matrix). */
static void or_solve3(double M[3][3], cplx r[3], cplx x[3]) {
    double A[3][3];
    cplx b[3];
    memcpy(A, M, sizeof(A));
    for (int i = 0; i < 3; ++i) b[i] = r[i];
    for (int c = 0; c < 3; ++c) {
        int piv = c;
        for (int i = c + 1; i < 3; ++i)
            if (fabs(A[i][c]) > fabs(A[piv][c])) piv = i;
        if (piv != c) {
            for (int j = 0; j < 3; ++j) { double t = A[c][j]; A[c][j] = A[piv][j]; A[piv][j] = t; }
            cplx t = b[c]; b[c] = b[piv]; b[piv] = t;
        }
        for (int i = c + 1; i < 3; ++i) {
            double f = A[i][c] / A[c][c];
            for (int j = c; j < 3; ++j) A[i][j] -= f * A[c][j];
            b[i] -= f * b[c];
        }
    }
    for (int i = 2; i >= 0; --i) {
        cplx s = b[i];
        for (int j = i + 1; j < 3; ++j) s -= A[i][j] * x[j];
        x[i] = s / A[i][i];
    }
}

/* Apply beta*A (inverse = 0) or (beta*A)^{-1} (inverse = 1) to a vector field
 * wavenumber by wavenumber.  At k = 0 the symbol of beta*A is 0 and the inverse
 * is taken as the identity (the seminorm has constants in its null space). */
static void or_apply_symbol(int n1, int n2, int n3, double beta, double gamma,
                            const double *v, double *out, int inverse) {
    const int n[3] = {n1, n2, n3};
    long N = (long)n1 * n2 * n3;
    cplx *V[3], *W[3];
    for (int d = 0; d < 3; ++d) {
        V[d] = or_spectrum(n, v + d * N);
        W[d] = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    }
    #pragma omp parallel for collapse(2) schedule(static)
    for (int i1 = 0; i1 < n1; ++i1)
        for (int i2 = 0; i2 < n2; ++i2)
            for (int i3 = 0; i3 < n3; ++i3) {
                const int ii[3] = {i1, i2, i3};
                double k[3], kh[3], M[3][3];
                for (int d = 0; d < 3; ++d) {
                    k[d] = or_wavenumber(ii[d], n[d]);
                    kh[d] = or_wavenumber_d1(ii[d], n[d]);
                }
                long id = or_idx(n, i1, i2, i3);
                cplx r[3], x[3];
                for (int d = 0; d < 3; ++d) r[d] = V[d][id];
                or_symbol_A(beta, gamma, k, kh, M);
                int zero_mode = (i1 == 0 && i2 == 0 && i3 == 0);
                if (!inverse) {
                    for (int a = 0; a < 3; ++a) {
                        x[a] = 0;
                        for (int b = 0; b < 3; ++b) x[a] += M[a][b] * r[b];
                    }
                } else if (zero_mode) {
                    for (int a = 0; a < 3; ++a) x[a] = r[a];
                } else {
                    or_solve3(M, r, x);
                }
                for (int d = 0; d < 3; ++d) W[d][id] = x[d];
            }
    for (int d = 0; d < 3; ++d) {
        or_field(n, W[d], out + d * N);
        free(W[d]);
        free(V[d]);
    }
}

void or_apply_A(int n1, int n2, int n3, double beta, double gamma, const double *v, double *out) {
    or_apply_symbol(n1, n2, n3, beta, gamma, v, out, 0);
}

void or_apply_Ainv(int n1, int n2, int n3, double beta, double gamma, const double *v, double *out) {
    or_apply_symbol(n1, n2, n3, beta, gamma, v, out, 1);
}

/* ------------------------------------------------------------------------- */
/* Periodic cubic Lagrange interpolation (Section 4.1)                         */
/*   f(q) = sum_{a,b,c} f[i0+a, j0+b, k0+c] phi_a(t1) phi_b(t2) phi_c(t3)     */
/* with nodes a in {-1, 0, 1, 2} around i0 = floor(q), t = q - i0.             */
/* ------------------------------------------------------------------------- */

/* Lagrange basis polynomial of node a (a in -1..2) on the nodes -1,0,1,2 */
double or_lagrange(int a, double t) {
    double p = 1.0;
    for (int b = -1; b <= 2; ++b)
        if (b != a) p *= (t - (double)b) / (double)(a - b);
    return p;
}

/* value of the periodic cubic interpolant of f at index-space point q */
static double or_interp_at(const int n[3], const double *f, const double q[3]) {
    long base[3];
    double w[3][4];
    for (int d = 0; d < 3; ++d) {
        double fl = floor(q[d]);
        double t = q[d] - fl;
        base[d] = (long)fl;
        for (int a = -1; a <= 2; ++a) w[d][a + 1] = or_lagrange(a, t);
    }
    double s = 0.0;
    for (int a = -1; a <= 2; ++a)
        for (int b = -1; b <= 2; ++b)
            for (int c = -1; c <= 2; ++c) {
                long i1 = or_wrap(base[0] + a, n[0]);
                long i2 = or_wrap(base[1] + b, n[1]);
                long i3 = or_wrap(base[2] + c, n[2]);
                s += f[or_idx(n, i1, i2, i3)] * w[0][a + 1] * w[1][b + 1] * w[2][c + 1];
            }
    return s;
}

/* interpolate f at npts points given in index units (q_d[p]) */
void or_interp(int n1, int n2, int n3, const double *f, long npts,
               const double *q1, const double *q2, const double *q3, double *out) {
    const int n[3] = {n1, n2, n3};
    #pragma omp parallel for schedule(static)
    for (long p = 0; p < npts; ++p) {
        double q[3] = {q1[p], q2[p], q3[p]};
        out[p] = or_interp_at(n, f, q);
    }
}

double or_lerp_at(const int n[3], const double *f, const double q[3]);
void or_grad_fd8(int n1, int n2, int n3, const double *f, double *g);
void or_div_fd8(int n1, int n2, int n3, const double *v, double *out);

/* interpolant of the given order: 3 = cubic Lagrange, 1 = trilinear */
static double or_interp_o(int order, const int n[3], const double *f, const double q[3]) {
    return order == 1 ? or_lerp_at(n, f, q) : or_interp_at(n, f, q);
}

/* interpolate f at the foot points of all grid points: the foot point of grid
 * point (i1,i2,i3) is (i1,i2,i3) + disp(i1,i2,i3) in index units */
static void or_interp_grid_o(int order, const int n[3], const double *f, const double *disp,
                             double *out) {
    long N = (long)n[0] * n[1] * n[2];
    #pragma omp parallel for collapse(2) schedule(static)
    for (int i1 = 0; i1 < n[0]; ++i1)
        for (int i2 = 0; i2 < n[1]; ++i2)
            for (int i3 = 0; i3 < n[2]; ++i3) {
                long id = or_idx(n, i1, i2, i3);
                double q[3] = {i1 + disp[id], i2 + disp[N + id], i3 + disp[2 * N + id]};
                out[id] = or_interp_o(order, n, f, q);
            }
}

/* ------------------------------------------------------------------------- */
/* Characteristics (Section 3 "Discretization"): dy/dt = v(y) on [t, t+dt],    */
/* y(t+dt) = x, by a second-order Runge-Kutta (Heun) step.                     */
/*   backward foot point (state):   X-(x) = x - dt/2 [v(x) + v(x - dt v(x))]   */
/*   forward foot point (adjoint):  X+(x) = x + dt/2 [v(x) + v(x + dt v(x))]   */
/* v is in domain units; the result is the displacement X - x in index units.  */
/* sign = -1 gives X-, sign = +1 gives X+.                                     */
/* ------------------------------------------------------------------------- */
static void or_footpoints_o(int order, int n1, int n2, int n3, int nt, const double *v, int sign,
                            double *disp) {
    const int n[3] = {n1, n2, n3};
    long N = (long)n1 * n2 * n3;
    double dt = 1.0 / nt;
    double h[3] = {2 * OR_PI / n1, 2 * OR_PI / n2, 2 * OR_PI / n3};
    #pragma omp parallel for collapse(2) schedule(static)
    for (int i1 = 0; i1 < n1; ++i1)
        for (int i2 = 0; i2 < n2; ++i2)
            for (int i3 = 0; i3 < n3; ++i3) {
                long id = or_idx(n, i1, i2, i3);
                const int ii[3] = {i1, i2, i3};
                double vx[3], ystar[3], vy[3];
                for (int d = 0; d < 3; ++d) vx[d] = v[d * N + id];
                /* predictor (explicit Euler), in index units */
                for (int d = 0; d < 3; ++d) ystar[d] = ii[d] + sign * dt * vx[d] / h[d];
                for (int d = 0; d < 3; ++d) vy[d] = or_interp_o(order, n, v + d * N, ystar);
                /* corrector (trapezoid) */
                for (int d = 0; d < 3; ++d)
                    disp[d * N + id] = sign * 0.5 * dt * (vx[d] + vy[d]) / h[d];
            }
}

void or_footpoints(int n1, int n2, int n3, int nt, const double *v, int sign, double *disp) {
    or_footpoints_o(3, n1, n2, n3, nt, v, sign, disp);
}

/* ------------------------------------------------------------------------- */
/* Transport solves                                                           */
/* ------------------------------------------------------------------------- */

/* trapezoidal quadrature weight of time level j of 0..nt */
static double or_trap_w(int j, int nt) { return (j == 0 || j == nt) ? 0.5 : 1.0; }

/* state equation (Eq. 2.1b): d_t m + v.grad m = 0, m(0) = m0.
 * Semi-Lagrangian: m^{j+1}(x) = m^j(X-(x)).  mhist holds m^0..m^nt. */
static void or_state_o(int order, int n1, int n2, int n3, int nt, const double *dispm,
                       const double *m0, double *mhist) {
    const int n[3] = {n1, n2, n3};
    long N = (long)n1 * n2 * n3;
    memcpy(mhist, m0, sizeof(double) * (size_t)N);
    for (int j = 0; j < nt; ++j)
        or_interp_grid_o(order, n, mhist + (long)j * N, dispm, mhist + (long)(j + 1) * N);
}
void or_state(int n1, int n2, int n3, int nt, const double *dispm, const double *m0, double *mhist) {
    or_state_o(3, n1, n2, n3, nt, dispm, m0, mhist);
}

/* Adjoint-type equation (Eqs. (3.2) and (3.6)): -d_t l - div(l v) = 0,
 * l(1) = lfinal, solved backward in time.  In reversed time s = 1 - t this is
 * d_s l - v.grad l = l div v, transport along -v with a source l*div(v).
 * Along the characteristic ending at x (foot point X+):
 *   predictor:  l*       = l^j(X+) + dt * l^j(X+) d(X+)
 *   corrector:  l^{j-1}(x) = l^j(X+) + dt/2 [ l^j(X+) d(X+) + l* d(x) ]
 * d = div v on the grid, dp = d interpolated at X+.  lhist holds l^0..l^nt. */
static void or_adjoint_o(int order, int n1, int n2, int n3, int nt, const double *dispp,
                         const double *d, const double *dp, const double *lfinal, double *lhist) {
    const int n[3] = {n1, n2, n3};
    long N = (long)n1 * n2 * n3;
    double dt = 1.0 / nt;
    double *lx = (double *)malloc(sizeof(double) * (size_t)N);
    memcpy(lhist + (long)nt * N, lfinal, sizeof(double) * (size_t)N);
    for (int j = nt; j >= 1; --j) {
        or_interp_grid_o(order, n, lhist + (long)j * N, dispp, lx);
        double *out = lhist + (long)(j - 1) * N;
        #pragma omp parallel for schedule(static)
        for (long i = 0; i < N; ++i) {
            double src0 = lx[i] * dp[i];
            double lstar = lx[i] + dt * src0;
            out[i] = lx[i] + 0.5 * dt * (src0 + lstar * d[i]);
        }
    }
    free(lx);
}

/* incremental state equation (Eq. 3.5): d_t mt + v.grad mt = f,
 * f = -vt.grad m, mt(0) = 0.  Along the characteristic ending at x
 * (foot point X-), trapezoid for the source:
 *   mt^{j+1}(x) = mt^j(X-) + dt/2 [ f^j(X-) + f^{j+1}(x) ].
 * gmhist holds grad m^j (3N per level).  mthist holds mt^0..mt^nt. */
static void or_incstate_o(int order, int n1, int n2, int n3, int nt, const double *dispm,
                          const double *gmhist, const double *vt, double *mthist) {
    const int n[3] = {n1, n2, n3};
    long N = (long)n1 * n2 * n3;
    double dt = 1.0 / nt;
    double *f = (double *)malloc(sizeof(double) * (size_t)N * (nt + 1));
    for (int j = 0; j <= nt; ++j) {
        const double *gm = gmhist + (long)j * 3 * N;
        for (long i = 0; i < N; ++i)
            f[(long)j * N + i] = -(vt[i] * gm[i] + vt[N + i] * gm[N + i] + vt[2 * N + i] * gm[2 * N + i]);
    }
    double *a = (double *)malloc(sizeof(double) * (size_t)N);
    double *b = (double *)malloc(sizeof(double) * (size_t)N);
    memset(mthist, 0, sizeof(double) * (size_t)N);
    for (int j = 0; j < nt; ++j) {
        or_interp_grid_o(order, n, mthist + (long)j * N, dispm, a);
        or_interp_grid_o(order, n, f + (long)j * N, dispm, b);
        double *out = mthist + (long)(j + 1) * N;
        #pragma omp parallel for schedule(static)
        for (long i = 0; i < N; ++i)
            out[i] = a[i] + 0.5 * dt * (b[i] + f[(long)(j + 1) * N + i]);
    }
    free(a);
    free(b);
    free(f);
}

void or_adjoint(int n1, int n2, int n3, int nt, const double *dispp, const double *d,
                const double *dp, const double *lfinal, double *lhist) {
    or_adjoint_o(3, n1, n2, n3, nt, dispp, d, dp, lfinal, lhist);
}
void or_incstate(int n1, int n2, int n3, int nt, const double *dispm, const double *gmhist,
                 const double *vt, double *mthist) {
    or_incstate_o(3, n1, n2, n3, nt, dispm, gmhist, vt, mthist);
}

/* body force (time integral in Eqs. (3.1) and (3.3)) by the trapezoidal rule:
 *   b = dt * sum_j w_j l^j grad m^j */
void or_bodyforce(long N, int nt, const double *lhist, const double *gmhist, double *b) {
    double dt = 1.0 / nt;
    memset(b, 0, sizeof(double) * (size_t)N * 3);
    for (int j = 0; j <= nt; ++j) {
        double w = dt * or_trap_w(j, nt);
        const double *l = lhist + (long)j * N;
        const double *gm = gmhist + (long)j * 3 * N;
        for (int d = 0; d < 3; ++d)
            for (long i = 0; i < N; ++i) b[d * N + i] += w * l[i] * gm[d * N + i];
    }
}

/* ------------------------------------------------------------------------- */
/* Problem object: images, parameters and the linearization at a velocity v    */
/* ------------------------------------------------------------------------- */
typedef struct {
    int n[3];
    long N;
    int nt;
    double beta, gamma;
    double *m0, *m1;
    /* linearization at v (valid when have_lin) */
    int have_lin;
    double *v;     /* 3N */
    double *dispm; /* 3N, X- - x */
    double *dispp; /* 3N, X+ - x */
    double *m;     /* (nt+1) N */
    double *gm;    /* (nt+1) 3N */
    double *d;     /* N, div v */
    double *dp;    /* N, div v at X+ */
    long n_pde;    /* transport solves done, for reports */
    int interp_order; /* 3: cubic Lagrange (default), 1: trilinear */
    int deriv_fd8;    /* 0: spectral first derivatives (default), 1: FD8 */
} or_problem;

/* discretization of the problem: interpolation order (3 or 1) and first
 * derivatives (0 spectral, 1 eighth-order finite differences) */
void or_set_discretization(or_problem *P, int interp_order, int deriv_fd8) {
    P->interp_order = interp_order == 1 ? 1 : 3;
    P->deriv_fd8 = deriv_fd8 ? 1 : 0;
    P->have_lin = 0;
}

static void or_grad_p(const or_problem *P, const double *f, double *g) {
    if (P->deriv_fd8) or_grad_fd8(P->n[0], P->n[1], P->n[2], f, g);
    else or_grad(P->n[0], P->n[1], P->n[2], f, g);
}
static void or_div_p(const or_problem *P, const double *v, double *out) {
    if (P->deriv_fd8) or_div_fd8(P->n[0], P->n[1], P->n[2], v, out);
    else or_div(P->n[0], P->n[1], P->n[2], v, out);
}

or_problem *or_create(int n1, int n2, int n3, int nt, double beta, double gamma,
                      const double *m0, const double *m1) {
    or_problem *P = (or_problem *)calloc(1, sizeof(or_problem));
    P->n[0] = n1; P->n[1] = n2; P->n[2] = n3;
    P->N = (long)n1 * n2 * n3;
    P->nt = nt;
    P->beta = beta;
    P->gamma = gamma;
    P->interp_order = 3;
    size_t N = (size_t)P->N;
    P->m0 = (double *)malloc(sizeof(double) * N);
    P->m1 = (double *)malloc(sizeof(double) * N);
    memcpy(P->m0, m0, sizeof(double) * N);
    memcpy(P->m1, m1, sizeof(double) * N);
    P->v = (double *)malloc(sizeof(double) * 3 * N);
    P->dispm = (double *)malloc(sizeof(double) * 3 * N);
    P->dispp = (double *)malloc(sizeof(double) * 3 * N);
    P->m = (double *)malloc(sizeof(double) * N * (nt + 1));
    P->gm = (double *)malloc(sizeof(double) * 3 * N * (nt + 1));
    P->d = (double *)malloc(sizeof(double) * N);
    P->dp = (double *)malloc(sizeof(double) * N);
    return P;
}

void or_destroy(or_problem *P) {
    if (!P) return;
    free(P->m0); free(P->m1); free(P->v); free(P->dispm); free(P->dispp);
    free(P->m); free(P->gm); free(P->d); free(P->dp);
    free(P);
}

static double or_h3(const or_problem *P) {
    return (2 * OR_PI / P->n[0]) * (2 * OR_PI / P->n[1]) * (2 * OR_PI / P->n[2]);
}

static double or_dot(long len, const double *a, const double *b) {
    double s = 0.0;
    for (long i = 0; i < len; ++i) s += a[i] * b[i];
    return s;
}

/* Linearize at v: foot points X- and X+, state m^j, grad m^j (stored, as in
 * Section 5.2 of the paper), d = div v and d(X+). */
void or_linearize(or_problem *P, const double *v) {
    int *n = P->n;
    long N = P->N;
    memcpy(P->v, v, sizeof(double) * 3 * N);
    const int o = P->interp_order;
    or_footpoints_o(o, n[0], n[1], n[2], P->nt, v, -1, P->dispm);
    or_footpoints_o(o, n[0], n[1], n[2], P->nt, v, +1, P->dispp);
    or_state_o(o, n[0], n[1], n[2], P->nt, P->dispm, P->m0, P->m);
    for (int j = 0; j <= P->nt; ++j) or_grad_p(P, P->m + (long)j * N, P->gm + (long)j * 3 * N);
    or_div_p(P, v, P->d);
    or_interp_grid_o(o, n, P->d, P->dispp, P->dp);
    P->have_lin = 1;
    P->n_pde += 1;
}

/* pointer to the linearization's m^j (for tests) */
const double *or_state_ptr(const or_problem *P) { return P->m; }
const double *or_gradstate_ptr(const or_problem *P) { return P->gm; }
const double *or_dispm_ptr(const or_problem *P) { return P->dispm; }
const double *or_dispp_ptr(const or_problem *P) { return P->dispp; }
const double *or_div_ptr(const or_problem *P) { return P->d; }
const double *or_divp_ptr(const or_problem *P) { return P->dp; }

/* objective J = 1/2 ||m(1) - m1||^2 + 1/2 <beta*A v, v>, L2 norms as h^3 sums.
 * Runs the state equation for v (does not change the stored linearization).
 * Returns J; *mismatch gets the first term, *regterm the second. */
double or_objective(or_problem *P, const double *v, double *mismatch, double *regterm,
                    double *m_final /* nullable, N */) {
    int *n = P->n;
    long N = P->N;
    double h3 = or_h3(P);
    double *dm = (double *)malloc(sizeof(double) * 3 * N);
    double *mh = (double *)malloc(sizeof(double) * N * (P->nt + 1));
    double *Av = (double *)malloc(sizeof(double) * 3 * N);
    or_footpoints_o(P->interp_order, n[0], n[1], n[2], P->nt, v, -1, dm);
    or_state_o(P->interp_order, n[0], n[1], n[2], P->nt, dm, P->m0, mh);
    const double *m1t = mh + (long)P->nt * N;
    double mis = 0.0;
    for (long i = 0; i < N; ++i) mis += (m1t[i] - P->m1[i]) * (m1t[i] - P->m1[i]);
    mis *= 0.5 * h3;
    or_apply_A(n[0], n[1], n[2], P->beta, P->gamma, v, Av);
    double reg = 0.5 * h3 * or_dot(3 * N, v, Av);
    if (m_final) memcpy(m_final, m1t, sizeof(double) * (size_t)N);
    free(dm); free(mh); free(Av);
    P->n_pde += 1;
    if (mismatch) *mismatch = mis;
    if (regterm) *regterm = reg;
    return mis + reg;
}

/* reduced gradient (Eq. 3.1): g = beta*A v + int_0^1 lambda grad m dt, with
 * the adjoint (Eq. 3.2) from lambda(1) = m1 - m(1).  Linearizes at v first.
 * Optionally returns J and the adjoint history (nt+1) N. */
void or_gradient(or_problem *P, const double *v, double *g, double *J, double *lhist_out) {
    int *n = P->n;
    long N = P->N;
    int nt = P->nt;
    or_linearize(P, v);
    double *lfinal = (double *)malloc(sizeof(double) * (size_t)N);
    double *lh = (double *)malloc(sizeof(double) * (size_t)N * (nt + 1));
    double *Av = (double *)malloc(sizeof(double) * 3 * (size_t)N);
    const double *mT = P->m + (long)nt * N;
    for (long i = 0; i < N; ++i) lfinal[i] = P->m1[i] - mT[i];
    or_adjoint_o(P->interp_order, n[0], n[1], n[2], nt, P->dispp, P->d, P->dp, lfinal, lh);
    or_bodyforce(N, nt, lh, P->gm, g);
    or_apply_A(n[0], n[1], n[2], P->beta, P->gamma, v, Av);
    for (long i = 0; i < 3 * N; ++i) g[i] += Av[i];
    if (J) {
        double h3 = or_h3(P);
        double mis = 0.5 * h3 * or_dot(N, lfinal, lfinal);
        *J = mis + 0.5 * h3 * or_dot(3 * N, v, Av);
    }
    if (lhist_out) memcpy(lhist_out, lh, sizeof(double) * (size_t)N * (nt + 1));
    free(lfinal); free(lh); free(Av);
    P->n_pde += 1;
}

/* Gauss-Newton Hessian matvec (Eq. 3.4): H vt = beta*A vt + int lt grad m dt,
 * lt from the incremental adjoint (Eq. 3.6) with lt(1) = -mt(1), mt from the
 * incremental state (Eq. 3.5).  Uses the stored linearization. Optionally
 * returns mt(1) (N) and the incremental adjoint history. */
int or_matvec(or_problem *P, const double *vt, double *Hvt, double *mt_final, double *lthist_out) {
    if (!P->have_lin) return 1;
    int *n = P->n;
    long N = P->N;
    int nt = P->nt;
    double *mth = (double *)malloc(sizeof(double) * (size_t)N * (nt + 1));
    double *lth = (double *)malloc(sizeof(double) * (size_t)N * (nt + 1));
    double *lfinal = (double *)malloc(sizeof(double) * (size_t)N);
    double *Av = (double *)malloc(sizeof(double) * 3 * (size_t)N);
    or_incstate_o(P->interp_order, n[0], n[1], n[2], nt, P->dispm, P->gm, vt, mth);
    for (long i = 0; i < N; ++i) lfinal[i] = -mth[(long)nt * N + i];
    or_adjoint_o(P->interp_order, n[0], n[1], n[2], nt, P->dispp, P->d, P->dp, lfinal, lth);
    or_bodyforce(N, nt, lth, P->gm, Hvt);
    or_apply_A(n[0], n[1], n[2], P->beta, P->gamma, vt, Av);
    for (long i = 0; i < 3 * N; ++i) Hvt[i] += Av[i];
    if (mt_final) memcpy(mt_final, mth + (long)nt * N, sizeof(double) * (size_t)N);
    if (lthist_out) memcpy(lthist_out, lth, sizeof(double) * (size_t)N * (nt + 1));
    free(mth); free(lth); free(lfinal); free(Av);
    P->n_pde += 2;
    return 0;
}

/* spectral preconditioner (Section 3 "Preconditioning"): s = (beta*A)^{-1} r */
void or_precond(or_problem *P, const double *r, double *s) {
    or_apply_Ainv(P->n[0], P->n[1], P->n[2], P->beta, P->gamma, r, s);
}

/* ------------------------------------------------------------------------- */
/* Preconditioned conjugate gradients (textbook Hestenes-Stiefel form)         */
/* ------------------------------------------------------------------------- */
typedef void (*or_op_fn)(void *ctx, const double *in, double *out);

/* Solve H x = b from x0 = 0.  Stops when ||r_i|| <= tol ||r_0|| (2-norms), or
 * after exactly maxit iterations if fixed != 0, or at maxit; on non-positive
 * curvature p.Hp <= 0 it stops and keeps the current iterate (the
 * preconditioned residual z0 if that happens in the first iteration).
 * Returns the number of iterations (matvecs); *flag = 0 ok, 1 neg. curvature,
 * 2 maxit reached without meeting tol (not set in fixed mode). */
long or_pcg_core(long len, or_op_fn H, void *Hctx, or_op_fn Pc, void *Pctx, const double *b,
                 double *x, double tol, long maxit, int fixed, int *flag, double *relres) {
    double *r = (double *)malloc(sizeof(double) * (size_t)len);
    double *z = (double *)malloc(sizeof(double) * (size_t)len);
    double *p = (double *)malloc(sizeof(double) * (size_t)len);
    double *q = (double *)malloc(sizeof(double) * (size_t)len);
    long it = 0;
    *flag = 0;
    for (long i = 0; i < len; ++i) { x[i] = 0.0; r[i] = b[i]; }
    double r0 = sqrt(or_dot(len, r, r));
    double rn = r0;
    if (r0 == 0.0) goto done;
    Pc(Pctx, r, z);
    for (long i = 0; i < len; ++i) p[i] = z[i];
    double rz = or_dot(len, r, z);
    while (it < maxit) {
        H(Hctx, p, q);
        double pq = or_dot(len, p, q);
        if (pq <= 0.0) {
            if (it == 0) for (long i = 0; i < len; ++i) x[i] = z[i];
            *flag = 1;
            ++it;
            break;
        }
        double alpha = rz / pq;
        for (long i = 0; i < len; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        ++it;
        rn = sqrt(or_dot(len, r, r));
        if (!fixed && rn <= tol * r0) break;
        if (it >= maxit) { if (!fixed) *flag = 2; break; }
        Pc(Pctx, r, z);
        double rz_new = or_dot(len, r, z);
        double beta = rz_new / rz;
        rz = rz_new;
        for (long i = 0; i < len; ++i) p[i] = z[i] + beta * p[i];
    }
done:
    if (relres) *relres = r0 > 0 ? rn / r0 : 0.0;
    free(r); free(z); free(p); free(q);
    return it;
}

/* dense-matrix operators, so the PCG routine itself can be checked against
 * a direct solve in the tests */
typedef struct { long n; const double *M; } or_dense;
static void or_dense_apply(void *c, const double *in, double *out) {
    or_dense *D = (or_dense *)c;
    for (long i = 0; i < D->n; ++i) {
        double s = 0.0;
        for (long j = 0; j < D->n; ++j) s += D->M[i * D->n + j] * in[j];
        out[i] = s;
    }
}

long or_pcg_dense(long n, const double *Hm, const double *Pm, const double *b, double *x,
                  double tol, long maxit, int fixed, int *flag, double *relres) {
    or_dense H = {n, Hm}, Pc = {n, Pm};
    return or_pcg_core(n, or_dense_apply, &H, or_dense_apply, &Pc, b, x, tol, maxit, fixed, flag,
                       relres);
}

static void or_matvec_cb(void *c, const double *in, double *out) {
    or_matvec((or_problem *)c, in, out, NULL, NULL);
}

long or_invh0(int n1, int n2, int n3, double beta0, double gamma, const double *gm,
              const double *r, double *s, double tol, long maxit);
long or_invh0_2l(int n1, int n2, int n3, double beta0, double gamma, const double *gm,
                 const double *r, double *s, double tol, long maxit);

/* outer preconditioner of the solver: InvA, InvH0 or two-level InvH0 with
 * grad m(1) of the current iterate and inner tolerance eps_h0 * eps_K */
typedef struct { or_problem *P; int pc; double tol; long maxit; long inner; } or_pc_ctx;
static void or_pc_cb(void *c, const double *in, double *out) {
    or_pc_ctx *q = (or_pc_ctx *)c;
    or_problem *P = q->P;
    if (q->pc == 0) { or_precond(P, in, out); return; }
    double beta0 = P->beta < 5e-2 ? 5e-2 : P->beta;
    const double *gm1 = P->gm + (long)P->nt * 3 * P->N;
    if (q->pc == 1)
        q->inner += or_invh0(P->n[0], P->n[1], P->n[2], beta0, P->gamma, gm1, in, out, q->tol, q->maxit);
    else
        q->inner += or_invh0_2l(P->n[0], P->n[1], P->n[2], beta0, P->gamma, gm1, in, out, q->tol, q->maxit);
}

/* ------------------------------------------------------------------------- */
/* Gauss-Newton-Krylov solver with Armijo line search (Algorithm 1, Eq. 3.3)   */
/* ------------------------------------------------------------------------- */
typedef struct {
    int max_gn;        /* max Gauss-Newton iterations */
    int max_pcg;       /* max PCG iterations per GN step */
    int fixed_pcg;     /* if > 0: exactly this many PCG iterations per GN step */
    double eps_n;      /* relative gradient stop, 5e-2 in Algorithm 1 */
    double armijo_c1;  /* sufficient decrease constant */
    int max_ls;        /* max step halvings */
    int pc;            /* 0: (beta A)^{-1}, 1: InvH0, 2: two-level InvH0 */
    double eps_h0;     /* inner tolerance factor (1e-3 for the NIREP runs) */
    int max_inner;     /* max inner PCG iterations */
} or_solve_opts;

typedef struct {
    int n_gn, n_pcg, n_matvec, n_precond, status;
    double J0, J, g0, g, grel, mismatch_rel;
    long n_inner;
} or_solve_report;

/* status: 0 converged (or max_gn / fixed work done), 1 line search failed */
int or_solve(or_problem *P, double *v, const or_solve_opts *o, or_solve_report *rep) {
    long N3 = 3 * P->N;
    double h3 = or_h3(P);
    double *g = (double *)malloc(sizeof(double) * (size_t)N3);
    double *rhs = (double *)malloc(sizeof(double) * (size_t)N3);
    double *vt = (double *)malloc(sizeof(double) * (size_t)N3);
    double *vn = (double *)malloc(sizeof(double) * (size_t)N3);
    memset(rep, 0, sizeof(*rep));
    double J;
    or_gradient(P, v, g, &J, NULL);
    double g0 = sqrt(or_dot(N3, g, g));
    rep->J0 = J;
    rep->g0 = g0;
    double gn = g0;
    int k = 0;
    for (;;) {
        double grel = g0 > 0 ? gn / g0 : 0.0;
        if (grel <= o->eps_n || k >= o->max_gn) break;
        /* inexact Newton forcing term (Algorithm 1) */
        double epsk = fmin(sqrt(grel), 0.5);
        for (long i = 0; i < N3; ++i) rhs[i] = -g[i];
        int flag;
        long maxit = o->fixed_pcg > 0 ? o->fixed_pcg : o->max_pcg;
        or_pc_ctx pcc = {P, o->pc, o->eps_h0 * epsk, o->max_inner, 0};
        long it = or_pcg_core(N3, or_matvec_cb, P, or_pc_cb, &pcc, rhs, vt, epsk, maxit,
                              o->fixed_pcg > 0, &flag, NULL);
        rep->n_inner += pcc.inner;
        rep->n_pcg += (int)it;
        rep->n_matvec += (int)it;
        rep->n_precond += (int)it;
        /* Armijo backtracking on J along vt */
        double slope = h3 * or_dot(N3, g, vt);
        double alpha = 1.0;
        int ok = 0;
        for (int ls = 0; ls <= o->max_ls; ++ls) {
            for (long i = 0; i < N3; ++i) vn[i] = v[i] + alpha * vt[i];
            double Jt = or_objective(P, vn, NULL, NULL, NULL);
            if (Jt <= J + o->armijo_c1 * alpha * slope) { ok = 1; break; }
            alpha *= 0.5;
        }
        if (!ok) { rep->status = 1; break; }
        memcpy(v, vn, sizeof(double) * (size_t)N3);
        ++k;
        or_gradient(P, v, g, &J, NULL);
        gn = sqrt(or_dot(N3, g, g));
    }
    rep->n_gn = k;
    rep->J = J;
    rep->g = gn;
    rep->grel = g0 > 0 ? gn / g0 : 0.0;
    {
        /* relative mismatch ||m(1) - m1|| / ||m0 - m1|| at the final v */
        long N = P->N;
        const double *mT = P->m + (long)P->nt * N;
        double a = 0, b = 0;
        for (long i = 0; i < N; ++i) {
            a += (mT[i] - P->m1[i]) * (mT[i] - P->m1[i]);
            b += (P->m0[i] - P->m1[i]) * (P->m0[i] - P->m1[i]);
        }
        rep->mismatch_rel = b > 0 ? sqrt(a / b) : 0.0;
    }
    free(g); free(rhs); free(vt); free(vn);
    return rep->status;
}

/* ------------------------------------------------------------------------- */
/* Diagnostic: determinant of the deformation gradient                         */
/* The backward map y with m(x,1) = m0(y(x)) is the composition of nt foot-    */
/* point maps X-.  Its displacement u = y - x obeys u^0 = 0,                   */
/*   u^{j+1}(x) = u^j(X-(x)) + (X-(x) - x),                                    */
/* and det grad y = det(Id + grad u) with the spectral gradient (u periodic).  */
/* Returned in index units per component for u, so grad is scaled by 1/h.      */
/* ------------------------------------------------------------------------- */
void or_det_grad_y(int n1, int n2, int n3, int nt, const double *v, double *det) {
    const int n[3] = {n1, n2, n3};
    long N = (long)n1 * n2 * n3;
    double h[3] = {2 * OR_PI / n1, 2 * OR_PI / n2, 2 * OR_PI / n3};
    double *dm = (double *)malloc(sizeof(double) * 3 * (size_t)N);
    double *u = (double *)calloc(3 * (size_t)N, sizeof(double));
    double *tmp = (double *)malloc(sizeof(double) * (size_t)N);
    double *G = (double *)malloc(sizeof(double) * 9 * (size_t)N);
    or_footpoints(n1, n2, n3, nt, v, -1, dm);
    for (int j = 0; j < nt; ++j)
        for (int d = 0; d < 3; ++d) {
            or_interp_grid_o(3, n, u + d * N, dm, tmp);
            for (long i = 0; i < N; ++i) u[d * N + i] = tmp[i] + dm[d * N + i];
        }
    /* u in domain units, then J_ab = delta_ab + d_b u_a */
    for (int d = 0; d < 3; ++d)
        for (long i = 0; i < N; ++i) u[d * N + i] *= h[d];
    for (int a = 0; a < 3; ++a) or_grad(n1, n2, n3, u + a * N, G + (long)a * 3 * N);
    for (long i = 0; i < N; ++i) {
        double J[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) J[a][b] = (a == b ? 1.0 : 0.0) + G[((long)a * 3 + b) * N + i];
        det[i] = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1])
               - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
               + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    }
    free(dm); free(u); free(tmp); free(G);
}

/* ------------------------------------------------------------------------- */
/* Zero-velocity Hessian preconditioners (Section 3 "Preconditioning",        */
/* Algorithm 2).                                                              */
/*   H0 s = beta0 A s + grad m (grad m . s),   beta0 = max(beta, 5e-2)        */
/* with grad m the gradient of the deformed template m(1) at the current      */
/* iterate.  InvH0 solves H0 s = r by PCG with preconditioner (beta0 A)^{-1}  */
/* from s = 0 to relative residual tol (the left-preconditioned system of     */
/* Algorithm 2 has the same solution).  The two-level variant solves the      */
/* same system on a grid of half the resolution for the restricted residual   */
/* and restricted grad m, prolongs the solution and adds the high-pass part   */
/* of (beta0 A)^{-1} r.                                                        */
/* ------------------------------------------------------------------------- */

void or_h0_matvec(int n1, int n2, int n3, double beta0, double gamma, const double *gm,
                  const double *s, double *out) {
    long N = (long)n1 * n2 * n3;
    or_apply_A(n1, n2, n3, beta0, gamma, s, out);
    #pragma omp parallel for schedule(static)
    for (long i = 0; i < N; ++i) {
        double gs = gm[i] * s[i] + gm[N + i] * s[N + i] + gm[2 * N + i] * s[2 * N + i];
        for (int d = 0; d < 3; ++d) out[d * N + i] += gm[d * N + i] * gs;
    }
}

typedef struct { int n[3]; double beta0, gamma; const double *gm; } or_h0_ctx;
static void or_h0_cb(void *c, const double *in, double *out) {
    or_h0_ctx *h = (or_h0_ctx *)c;
    or_h0_matvec(h->n[0], h->n[1], h->n[2], h->beta0, h->gamma, h->gm, in, out);
}
static void or_ainv_cb(void *c, const double *in, double *out) {
    or_h0_ctx *h = (or_h0_ctx *)c;
    or_apply_Ainv(h->n[0], h->n[1], h->n[2], h->beta0, h->gamma, in, out);
}

/* s = H0^{-1} r by PCG; returns the iteration count */
long or_invh0(int n1, int n2, int n3, double beta0, double gamma, const double *gm,
              const double *r, double *s, double tol, long maxit) {
    or_h0_ctx h = {{n1, n2, n3}, beta0, gamma, gm};
    int flag;
    return or_pcg_core(3L * n1 * n2 * n3, or_h0_cb, &h, or_ainv_cb, &h, r, s, tol, maxit, 0, &flag,
                       NULL);
}

/* Spectral restriction of a field on an n grid to an nc grid (nc <= n per
 * axis): keep the wavenumbers with |k_d| < nc_d/2 (the coarse Nyquist mode is
 * dropped), rescale for the coarse transform length. */
void or_restrict(const int n[3], const int nc[3], const double *f, double *fc) {
    long N = (long)n[0] * n[1] * n[2], Nc = (long)nc[0] * nc[1] * nc[2];
    cplx *F = or_spectrum(n, f);
    cplx *G = (cplx *)calloc((size_t)Nc, sizeof(cplx));
    for (int i1 = 0; i1 < nc[0]; ++i1)
        for (int i2 = 0; i2 < nc[1]; ++i2)
            for (int i3 = 0; i3 < nc[2]; ++i3) {
                const int ic[3] = {i1, i2, i3};
                long src[3];
                int keep = 1;
                for (int d = 0; d < 3; ++d) {
                    double k = or_wavenumber(ic[d], nc[d]);
                    if (2.0 * fabs(k) >= nc[d]) keep = 0;
                    src[d] = k < 0 ? (long)(n[d] + k) : (long)k;
                }
                if (keep) G[or_idx(nc, i1, i2, i3)] = F[or_idx(n, src[0], src[1], src[2])] * ((double)Nc / (double)N);
            }
    or_field(nc, G, fc);
    free(F);
    free(G);
}

/* Spectral prolongation from an nc grid to an n grid: the coarse wavenumbers
 * with |k_d| < nc_d/2 are placed into the fine spectrum (zero elsewhere). */
void or_prolong(const int nc[3], const int n[3], const double *fc, double *f) {
    long N = (long)n[0] * n[1] * n[2], Nc = (long)nc[0] * nc[1] * nc[2];
    cplx *G = or_spectrum(nc, fc);
    cplx *F = (cplx *)calloc((size_t)N, sizeof(cplx));
    for (int i1 = 0; i1 < nc[0]; ++i1)
        for (int i2 = 0; i2 < nc[1]; ++i2)
            for (int i3 = 0; i3 < nc[2]; ++i3) {
                const int ic[3] = {i1, i2, i3};
                long dst[3];
                int keep = 1;
                for (int d = 0; d < 3; ++d) {
                    double k = or_wavenumber(ic[d], nc[d]);
                    if (2.0 * fabs(k) >= nc[d]) keep = 0;
                    dst[d] = k < 0 ? (long)(n[d] + k) : (long)k;
                }
                if (keep) F[or_idx(n, dst[0], dst[1], dst[2])] = G[or_idx(nc, i1, i2, i3)] * ((double)N / (double)Nc);
            }
    or_field(n, F, f);
    free(F);
    free(G);
}

/* the part of f that the half grid does not represent: f - P(R(f)) */
void or_highpass(const int n[3], const int nc[3], const double *f, double *out) {
    long N = (long)n[0] * n[1] * n[2], Nc = (long)nc[0] * nc[1] * nc[2];
    double *c = (double *)malloc(sizeof(double) * (size_t)Nc);
    or_restrict(n, nc, f, c);
    or_prolong(nc, n, c, out);
    for (long i = 0; i < N; ++i) out[i] = f[i] - out[i];
    free(c);
}

/* two-level InvH0 (Algorithm 2, second function); returns coarse iterations */
long or_invh0_2l(int n1, int n2, int n3, double beta0, double gamma, const double *gm,
                 const double *r, double *s, double tol, long maxit) {
    const int n[3] = {n1, n2, n3};
    const int nc[3] = {n1 / 2, n2 / 2, n3 / 2};
    long N = (long)n1 * n2 * n3, Nc = (long)nc[0] * nc[1] * nc[2];
    double *sf = (double *)malloc(sizeof(double) * 3 * (size_t)N);
    double *hp = (double *)malloc(sizeof(double) * 3 * (size_t)N);
    double *rc = (double *)malloc(sizeof(double) * 3 * (size_t)Nc);
    double *gmc = (double *)malloc(sizeof(double) * 3 * (size_t)Nc);
    double *sc = (double *)malloc(sizeof(double) * 3 * (size_t)Nc);
    or_apply_Ainv(n1, n2, n3, beta0, gamma, r, sf);
    for (int d = 0; d < 3; ++d) {
        or_highpass(n, nc, sf + d * N, hp + d * N);
        or_restrict(n, nc, r + d * N, rc + d * Nc);
        or_restrict(n, nc, gm + d * N, gmc + d * Nc);
    }
    long it = or_invh0(nc[0], nc[1], nc[2], beta0, gamma, gmc, rc, sc, tol, maxit);
    for (int d = 0; d < 3; ++d) {
        or_prolong(nc, n, sc + d * Nc, s + d * N);
        for (long i = 0; i < N; ++i) s[d * N + i] += hp[d * N + i];
    }
    free(sf); free(hp); free(rc); free(gmc); free(sc);
    return it;
}

/* ------------------------------------------------------------------------- */
/* Parameter continuation in beta (Section 3 "Preconditioning", last          */
/* paragraph): solve for beta_k = max(beta_target, beta_start * factor^k),    */
/* k = 0, 1, ..., each level started from the previous velocity; the spectral */
/* preconditioner is used while beta_k > 5e-1, the selected zero-velocity     */
/* preconditioner (o->pc) below.  Returns the status of the last level; the   */
/* report accumulates counts and holds the last level's values.               */
/* ------------------------------------------------------------------------- */
int or_solve_continuation(or_problem *P, double *v, double beta_target, double beta_start,
                          double factor, const or_solve_opts *o, or_solve_report *rep, int *levels) {
    or_solve_report r, acc;
    memset(&acc, 0, sizeof(acc));
    double b = beta_start > beta_target ? beta_start : beta_target;
    int nlev = 0, status = 0;
    for (;;) {
        or_solve_opts ol = *o;
        if (b > 5e-1) ol.pc = 0;
        P->beta = b;
        P->have_lin = 0;
        status = or_solve(P, v, &ol, &r);
        ++nlev;
        acc.n_gn += r.n_gn;
        acc.n_pcg += r.n_pcg;
        acc.n_matvec += r.n_matvec;
        acc.n_precond += r.n_precond;
        acc.n_inner += r.n_inner;
        if (nlev == 1) { acc.J0 = r.J0; acc.g0 = r.g0; }
        acc.J = r.J; acc.g = r.g; acc.grel = r.grel; acc.mismatch_rel = r.mismatch_rel;
        if (status != 0 || b <= beta_target) break;
        b = b * factor;
        if (b <= beta_target * (1.0 + 1e-9)) b = beta_target;  /* land exactly on the target */
    }
    acc.status = status;
    *rep = acc;
    if (levels) *levels = nlev;
    return status;
}

/* ------------------------------------------------------------------------- */
/* The paper's GPU discretization options (Sections 4.1, 4.2): eighth-order   */
/* central finite differences for first derivatives and trilinear             */
/* interpolation.  Selected per problem with or_set_discretization.           */
/* ------------------------------------------------------------------------- */

/* d/dx of a periodic line sample by the 8th-order central difference:
 * f'(x) ~ (1/h) sum_{j=1..4} c_j (f(x + j h) - f(x - j h)),
 * c = (4/5, -1/5, 4/105, -1/280) */
static const double or_fd8_c[4] = {4.0 / 5.0, -1.0 / 5.0, 4.0 / 105.0, -1.0 / 280.0};

void or_grad_fd8(int n1, int n2, int n3, const double *f, double *g) {
    const int n[3] = {n1, n2, n3};
    long N = (long)n1 * n2 * n3;
    #pragma omp parallel for collapse(2) schedule(static)
    for (int i1 = 0; i1 < n1; ++i1)
        for (int i2 = 0; i2 < n2; ++i2)
            for (int i3 = 0; i3 < n3; ++i3) {
                const int ii[3] = {i1, i2, i3};
                long id = or_idx(n, i1, i2, i3);
                for (int d = 0; d < 3; ++d) {
                    double h = 2 * OR_PI / n[d], s = 0.0;
                    for (int j = 1; j <= 4; ++j) {
                        int ip[3] = {i1, i2, i3}, im[3] = {i1, i2, i3};
                        ip[d] = (int)or_wrap(ii[d] + j, n[d]);
                        im[d] = (int)or_wrap(ii[d] - j, n[d]);
                        s += or_fd8_c[j - 1] * (f[or_idx(n, ip[0], ip[1], ip[2])] - f[or_idx(n, im[0], im[1], im[2])]);
                    }
                    g[d * N + id] = s / h;
                }
            }
}

void or_div_fd8(int n1, int n2, int n3, const double *v, double *out) {
    long N = (long)n1 * n2 * n3;
    double *g = (double *)malloc(sizeof(double) * 3 * (size_t)N);
    for (long i = 0; i < N; ++i) out[i] = 0.0;
    for (int d = 0; d < 3; ++d) {
        or_grad_fd8(n1, n2, n3, v + d * N, g);
        for (long i = 0; i < N; ++i) out[i] += g[d * N + i];
    }
    free(g);
}

/* trilinear (first-order Lagrange) periodic interpolation at index point q */
double or_lerp_at(const int n[3], const double *f, const double q[3]) {
    long base[3];
    double t[3];
    for (int d = 0; d < 3; ++d) {
        double fl = floor(q[d]);
        base[d] = (long)fl;
        t[d] = q[d] - fl;
    }
    double s = 0.0;
    for (int a = 0; a <= 1; ++a)
        for (int b = 0; b <= 1; ++b)
            for (int c = 0; c <= 1; ++c) {
                double w = (a ? t[0] : 1 - t[0]) * (b ? t[1] : 1 - t[1]) * (c ? t[2] : 1 - t[2]);
                s += w * f[or_idx(n, or_wrap(base[0] + a, n[0]), or_wrap(base[1] + b, n[1]),
                                  or_wrap(base[2] + c, n[2]))];
            }
    return s;
}

void or_lerp(int n1, int n2, int n3, const double *f, long npts, const double *q1,
             const double *q2, const double *q3, double *out) {
    const int n[3] = {n1, n2, n3};
    #pragma omp parallel for schedule(static)
    for (long p = 0; p < npts; ++p) {
        double q[3] = {q1[p], q2[p], q3[p]};
        out[p] = or_lerp_at(n, f, q);
    }
}
