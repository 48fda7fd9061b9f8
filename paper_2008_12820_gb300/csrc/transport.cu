// transport.cu -- semi-Lagrangian transport kernels (paper Section 3,
// "Discretization"; Section 4.1 interpolation).
//
// Every time step of every transport solve is one gather: the new value at
// grid point x is the old field interpolated (periodic cubic Lagrange, 4x4x4
// stencil around floor(x + disp)) at the foot point x + disp(x) of the
// characteristic through x, plus a pointwise epilogue that depends on the
// equation:
//   state (Eq. 2.1b)               m^{j+1}   = m^j(X-)
//   adjoint (Eq. 3.2, 3.6)         l^{j-1}   = c * l^j(X+)
//   incremental state (Eq. 3.5)    u^{j+1}   = u^j(X-) + dt f^{j+1},
//                                   f = -vt . grad m,  u = mt + dt/2 f
// The foot points are stored as displacements in grid-index units, so the
// integer part and the interpolation weight of each axis come from a small
// number (no loss of precision at large grid indices).
//
// One thread computes one output voxel; a block covers 32 consecutive x3
// points of 8 consecutive x2 rows, so the 64 gathers of a warp fall on a few
// cache lines of the same rows (the displacement field is smooth).
#include <cuda_runtime.h>

#include "claire_internal.cuh"

namespace claire {

namespace {

constexpr int BX = 32, BY = 8;

// cubic Lagrange basis on the nodes -1, 0, 1, 2 evaluated at t in [0, 1)
__device__ __forceinline__ void lagrange4(float t, float w[4]) {
    const float tp1 = t + 1.f, tm1 = t - 1.f, tm2 = t - 2.f;
    const float a = t * tm2;   // t (t - 2)
    const float b = tp1 * tm1; // (t + 1)(t - 1)
    w[0] = -(1.f / 6.f) * a * tm1;
    w[1] = 0.5f * b * tm2;
    w[2] = -0.5f * tp1 * a;
    w[3] = (1.f / 6.f) * b * t;
}

__device__ __forceinline__ int wrap_index(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// stencil of one axis: 4 wrapped node offsets (times the axis stride) and weights
struct Axis4 {
    int o[4];
    float w[4];
};

__device__ __forceinline__ void axis_stencil(int i, float disp, int n, int stride, Axis4 &a) {
    float fl = floorf(disp);
    // keep the integer conversion in range whatever the displacement
    fl = fminf(fmaxf(fl, -1.0e6f), 1.0e6f);
    lagrange4(disp - fl, a.w);
    int b = wrap_index(i + (int)fl - 1, n);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        a.o[k] = b * stride;
        b = (b + 1 == n) ? 0 : b + 1;
    }
}

__device__ __forceinline__ float gather64(const float *__restrict__ f, const Axis4 &a1,
                                          const Axis4 &a2, const Axis4 &a3) {
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float s2 = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float *row = f + a1.o[i] + a2.o[j];
            float s3 = a3.w[0] * __ldg(row + a3.o[0]);
            s3 = fmaf(a3.w[1], __ldg(row + a3.o[1]), s3);
            s3 = fmaf(a3.w[2], __ldg(row + a3.o[2]), s3);
            s3 = fmaf(a3.w[3], __ldg(row + a3.o[3]), s3);
            s2 = fmaf(a2.w[j], s3, s2);
        }
        acc = fmaf(a1.w[i], s2, acc);
    }
    return acc;
}

struct Pt {
    int i1, i2, i3;
    long long id;
    bool ok;
};

__device__ __forceinline__ Pt this_point(const Dims &d) {
    Pt p;
    p.i3 = blockIdx.x * BX + threadIdx.x;
    p.i2 = blockIdx.y * BY + threadIdx.y;
    p.i1 = blockIdx.z;
    p.ok = (p.i3 < d.n3) && (p.i2 < d.n2);
    p.id = ((long long)p.i1 * d.n2 + p.i2) * d.n3 + p.i3;
    return p;
}

__device__ __forceinline__ float interp_at(const float *__restrict__ f, const Dims &d, const Pt &p,
                                           float d1, float d2, float d3) {
    Axis4 a1, a2, a3;
    axis_stencil(p.i1, d1, d.n1, d.n2 * d.n3, a1);
    axis_stencil(p.i2, d2, d.n2, d.n3, a2);
    axis_stencil(p.i3, d3, d.n3, 1, a3);
    return gather64(f, a1, a2, a3);
}

// ---------------------------------------------------------------------------
// foot points: Heun (RK2) backward (sign -1) and forward (sign +1) in one pass
//   y* = x + s dt v(x);  X = x + s dt/2 (v(x) + v(y*));  disp = (X - x)/h
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(BX * BY)
k_footpoints(const float *__restrict__ v, float *__restrict__ dispm, float *__restrict__ dispp,
             Dims d, float dt, float ih1, float ih2, float ih3) {
    Pt p = this_point(d);
    if (!p.ok) return;
    const long long N = d.N;
    const float v1 = v[p.id], v2 = v[N + p.id], v3 = v[2 * N + p.id];
    const int nsides = dispp ? 2 : 1;  // X+ is skipped when not wanted
    for (int s = 0; s < nsides; ++s) {
        const float sg = s == 0 ? -1.f : 1.f;
        const float q1 = sg * dt * v1 * ih1, q2 = sg * dt * v2 * ih2, q3 = sg * dt * v3 * ih3;
        Axis4 a1, a2, a3;
        axis_stencil(p.i1, q1, d.n1, d.n2 * d.n3, a1);
        axis_stencil(p.i2, q2, d.n2, d.n3, a2);
        axis_stencil(p.i3, q3, d.n3, 1, a3);
        const float w1 = gather64(v, a1, a2, a3);
        const float w2 = gather64(v + N, a1, a2, a3);
        const float w3 = gather64(v + 2 * N, a1, a2, a3);
        float *out = s == 0 ? dispm : dispp;
        const float hs = 0.5f * sg * dt;
        out[p.id] = hs * (v1 + w1) * ih1;
        out[N + p.id] = hs * (v2 + w2) * ih2;
        out[2 * N + p.id] = hs * (v3 + w3) * ih3;
    }
}

// plain interpolation of f at x + disp
__global__ void __launch_bounds__(BX * BY)
k_interp(const float *__restrict__ f, const float *__restrict__ disp, float *__restrict__ out,
         Dims d) {
    Pt p = this_point(d);
    if (!p.ok) return;
    const long long N = d.N;
    out[p.id] = interp_at(f, d, p, disp[p.id], disp[N + p.id], disp[2 * N + p.id]);
}

// adjoint source factor along the forward characteristic (Heun for
// dl/ds = l div v):  c = 1 + dt/2 (d(X+) + d(x)) + dt^2/2 d(x) d(X+)
__global__ void __launch_bounds__(BX * BY)
k_adjoint_factor(const float *__restrict__ divv, const float *__restrict__ dispp,
                 float *__restrict__ cfac, Dims d, float dt) {
    Pt p = this_point(d);
    if (!p.ok) return;
    const long long N = d.N;
    const float dx = divv[p.id];
    const float dX = interp_at(divv, d, p, dispp[p.id], dispp[N + p.id], dispp[2 * N + p.id]);
    cfac[p.id] = 1.f + 0.5f * dt * (dX + dx) + 0.5f * dt * dt * dx * dX;
}

// state step: dst = src(X-)
__global__ void __launch_bounds__(BX * BY)
k_state_step(const float *__restrict__ src, const float *__restrict__ disp, float *__restrict__ dst,
             Dims d) {
    Pt p = this_point(d);
    if (!p.ok) return;
    const long long N = d.N;
    dst[p.id] = interp_at(src, d, p, disp[p.id], disp[N + p.id], disp[2 * N + p.id]);
}

// adjoint step: dst = c * src(X+)
__global__ void __launch_bounds__(BX * BY)
k_adjoint_step(const float *__restrict__ src, const float *__restrict__ disp,
               const float *__restrict__ cfac, float *__restrict__ dst, Dims d) {
    Pt p = this_point(d);
    if (!p.ok) return;
    const long long N = d.N;
    const float val = interp_at(src, d, p, disp[p.id], disp[N + p.id], disp[2 * N + p.id]);
    dst[p.id] = cfac[p.id] * val;
}

// incremental state step: dst = src(X-) + dt f^{j+1},  f = -vt . grad m^{j+1}
__global__ void __launch_bounds__(BX * BY)
k_incstate_step(const float *__restrict__ src, const float *__restrict__ disp,
                const float *__restrict__ vt, const float *__restrict__ gm, float *__restrict__ dst,
                Dims d, float dt) {
    Pt p = this_point(d);
    if (!p.ok) return;
    const long long N = d.N;
    const float val = interp_at(src, d, p, disp[p.id], disp[N + p.id], disp[2 * N + p.id]);
    const float f = -(vt[p.id] * gm[p.id] + vt[N + p.id] * gm[N + p.id] +
                      vt[2 * N + p.id] * gm[2 * N + p.id]);
    dst[p.id] = fmaf(dt, f, val);
}

// ----------------------------------------------------------- pointwise ----
constexpr int PT = 256;

__global__ void k_incstate_init(const float *__restrict__ vt, const float *__restrict__ gm,
                                float *__restrict__ u0, long long N, float hdt) {
    for (long long i = blockIdx.x * (long long)PT + threadIdx.x; i < N; i += (long long)gridDim.x * PT) {
        const float f = -(vt[i] * gm[i] + vt[N + i] * gm[N + i] + vt[2 * N + i] * gm[2 * N + i]);
        u0[i] = hdt * f;
    }
}

// lt(1) = -mt(1) = -(u^nt - dt/2 f^nt);  also returns mt(1)
__global__ void k_incadj_init(const float *__restrict__ u, const float *__restrict__ vt,
                              const float *__restrict__ gm, float *__restrict__ lt,
                              float *__restrict__ mt, long long N, float hdt) {
    for (long long i = blockIdx.x * (long long)PT + threadIdx.x; i < N; i += (long long)gridDim.x * PT) {
        const float f = -(vt[i] * gm[i] + vt[N + i] * gm[N + i] + vt[2 * N + i] * gm[2 * N + i]);
        const float m = u[i] - hdt * f;
        lt[i] = -m;
        if (mt) mt[i] = m;
    }
}

__global__ void k_sub(const float *__restrict__ a, const float *__restrict__ b,
                      float *__restrict__ out, long long N) {
    for (long long i = blockIdx.x * (long long)PT + threadIdx.x; i < N; i += (long long)gridDim.x * PT)
        out[i] = a[i] - b[i];
}

// body force by the trapezoidal rule: out_d = add_d + dt sum_j w_j l^j dm^j/dx_d
__global__ void k_bodyforce(const float *__restrict__ lh, const float *__restrict__ gmh,
                            const float *__restrict__ add, float *__restrict__ out, long long N,
                            int nt, float dt) {
    for (long long i = blockIdx.x * (long long)PT + threadIdx.x; i < N; i += (long long)gridDim.x * PT) {
        float b1 = 0.f, b2 = 0.f, b3 = 0.f;
        for (int j = 0; j <= nt; ++j) {
            const float w = (j == 0 || j == nt) ? 0.5f * dt : dt;
            const float l = w * lh[(long long)j * N + i];
            const float *g = gmh + (long long)j * 3 * N;
            b1 = fmaf(l, g[i], b1);
            b2 = fmaf(l, g[N + i], b2);
            b3 = fmaf(l, g[2 * N + i], b3);
        }
        if (add) {
            b1 += add[i];
            b2 += add[N + i];
            b3 += add[2 * N + i];
        }
        out[i] = b1;
        out[N + i] = b2;
        out[2 * N + i] = b3;
    }
}

inline dim3 grid3(const Dims &d) {
    return dim3((d.n3 + BX - 1) / BX, (d.n2 + BY - 1) / BY, d.n1);
}

inline int grid1(long long N) {
    long long b = (N + PT - 1) / PT;
    return (int)(b < 152 * 16 ? b : 152 * 16);
}

}  // namespace

void launch_footpoints(const Dims &d, int nt, const float *v, float *dispm, float *dispp,
                       cudaStream_t st, Profiler *prof) {
    const float dt = 1.f / nt;
    const double two_pi = 6.283185307179586476925286766559;
    ProfScope ps(prof, CLAIRE_K_FOOTPOINT, st, (double)d.N * (dispp ? 36 : 24));
    k_footpoints<<<grid3(d), dim3(BX, BY), 0, st>>>(v, dispm, dispp, d, dt,
                                                    (float)(d.n1 / two_pi), (float)(d.n2 / two_pi),
                                                    (float)(d.n3 / two_pi));
}

void launch_interp(const Dims &d, const float *f, const float *disp, float *out, cudaStream_t st,
                   Profiler *prof, int kclass) {
    ProfScope ps(prof, kclass, st, 20.0 * d.N);
    k_interp<<<grid3(d), dim3(BX, BY), 0, st>>>(f, disp, out, d);
}

void launch_adjoint_factor(const Dims &d, int nt, const float *divv, const float *dispp,
                           float *cfac, cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_FOOTPOINT, st, 20.0 * d.N);
    k_adjoint_factor<<<grid3(d), dim3(BX, BY), 0, st>>>(divv, dispp, cfac, d, 1.f / nt);
}

void launch_state_step(const Dims &d, const float *src, const float *dispm, float *dst,
                       cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_STATE, st, 20.0 * d.N);
    k_state_step<<<grid3(d), dim3(BX, BY), 0, st>>>(src, dispm, dst, d);
}

void launch_adjoint_step(const Dims &d, const float *src, const float *dispp, const float *cfac,
                         float *dst, cudaStream_t st, Profiler *prof, int kclass) {
    ProfScope ps(prof, kclass, st, 24.0 * d.N);
    k_adjoint_step<<<grid3(d), dim3(BX, BY), 0, st>>>(src, dispp, cfac, dst, d);
}

void launch_incstate_init(const Dims &d, float dt, const float *vt, const float *gm0, float *u0,
                          cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_VECTOR, st, 28.0 * d.N);
    k_incstate_init<<<grid1(d.N), PT, 0, st>>>(vt, gm0, u0, d.N, 0.5f * dt);
}

void launch_incstate_step(const Dims &d, float dt, const float *src, const float *dispm,
                          const float *vt, const float *gm_next, float *dst, cudaStream_t st,
                          Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_INCSTATE, st, 44.0 * d.N);
    k_incstate_step<<<grid3(d), dim3(BX, BY), 0, st>>>(src, dispm, vt, gm_next, dst, d, dt);
}

void launch_incadj_init(const Dims &d, float dt, const float *u_last, const float *vt,
                        const float *gm_last, float *lt_last, float *mt_out, cudaStream_t st,
                        Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_VECTOR, st, (double)d.N * (mt_out ? 36 : 32));
    k_incadj_init<<<grid1(d.N), PT, 0, st>>>(u_last, vt, gm_last, lt_last, mt_out, d.N, 0.5f * dt);
}

void launch_sub(const Dims &d, const float *a, const float *b, float *out, cudaStream_t st,
                Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_VECTOR, st, 12.0 * d.N);
    k_sub<<<grid1(d.N), PT, 0, st>>>(a, b, out, d.N);
}

void launch_bodyforce(const Dims &d, int nt, const float *lhist, const float *gmhist,
                      const float *add, float *out, cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_BODYFORCE, st, (double)d.N * (16.0 * (nt + 1) + 12 + (add ? 12 : 0)));
    k_bodyforce<<<grid1(d.N), PT, 0, st>>>(lhist, gmhist, add, out, d.N, nt, 1.f / nt);
}

}  // namespace claire
