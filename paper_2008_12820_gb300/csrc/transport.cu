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
// The time-step kernels stage the source field in shared-memory halo boxes
// (k_sl_tiled); the foot-point kernel gathers v from global memory, one
// thread per voxel, a block covering 32 consecutive x3 points of 8 x2 rows.
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
    // one period off is the common case; the modulo handles the rest
    if (i < 0) i += n;
    else if (i >= n) i -= n;
    if ((unsigned)i >= (unsigned)n) {
        i %= n;
        if (i < 0) i += n;
    }
    return i;
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

// ---------------------------------------------------------------------------
// Shared-memory tiled semi-Lagrangian step.
// A block owns T3 x T2 x T1 = 32 x 8 x 4 output voxels (a warp per x2 row,
// every thread 4 voxels along x1).  Per-step displacements are a few cells, so
// the 4x4x4 stencils of a block cover a small box of the source field: the
// block takes the minimum and maximum floor of its displacements per axis,
// stages that box in shared memory once (coalesced rows, periodic wrap) and
// reads the 64 taps of every output from there with immediate offsets.  A
// block whose box exceeds the capacity (large displacements) gathers from
// global memory instead; the choice is uniform over the block.
// ---------------------------------------------------------------------------
constexpr int T3 = 32, T2 = 8, T1 = 4;
constexpr int BOX_CAP = 8192;  // floats of shared memory for the box

enum SlMode { SL_PLAIN = 0, SL_ADJ = 1, SL_INCSTATE = 2, SL_ADJFAC = 3 };

struct SlArgs {
    const float *src;   // field gathered at the foot points
    const float *disp;  // foot point minus grid point, index units, [3][N]
    float *dst;
    const float *aux;   // SL_ADJ: c;  SL_ADJFAC: div v on the grid
    const float *vt;    // SL_INCSTATE: vt [3][N]
    const float *gm;    // SL_INCSTATE: grad m^{j+1} [3][N]
    float dt;
};

__device__ __forceinline__ int floor_int(float x) {
    return (int)fminf(fmaxf(floorf(x), -1.0e6f), 1.0e6f);
}

template <int MODE>
__global__ void __launch_bounds__(T3 * T2)
k_sl_tiled(SlArgs a, Dims d) {
    extern __shared__ float box[];
    __shared__ int fmin_s[3], fmax_s[3];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i3 = blockIdx.x * T3 + tx;
    const int i2 = blockIdx.y * T2 + ty;
    const int i1b = blockIdx.z * T1;
    const bool ok23 = (i3 < d.n3) && (i2 < d.n2);
    const long long N = d.N;
    if (ty == 0 && tx < 3) {
        fmin_s[tx] = 0x7fffffff;
        fmax_s[tx] = -0x7fffffff;
    }
    float dd[T1][3];
    int mn0 = 0x7fffffff, mn1 = 0x7fffffff, mn2 = 0x7fffffff;
    int mx0 = -0x7fffffff, mx1 = -0x7fffffff, mx2 = -0x7fffffff;
#pragma unroll
    for (int t = 0; t < T1; ++t) {
        const int i1 = i1b + t;
        if (ok23 && i1 < d.n1) {
            const long long id = ((long long)i1 * d.n2 + i2) * d.n3 + i3;
            dd[t][0] = a.disp[id];
            dd[t][1] = a.disp[N + id];
            dd[t][2] = a.disp[2 * N + id];
            const int f0 = floor_int(dd[t][0]), f1 = floor_int(dd[t][1]), f2 = floor_int(dd[t][2]);
            mn0 = min(mn0, f0); mx0 = max(mx0, f0);
            mn1 = min(mn1, f1); mx1 = max(mx1, f1);
            mn2 = min(mn2, f2); mx2 = max(mx2, f2);
        } else {
            dd[t][0] = dd[t][1] = dd[t][2] = 0.f;
        }
    }
    __syncthreads();  // fmin_s / fmax_s initialized
    mn0 = __reduce_min_sync(0xffffffffu, mn0); mx0 = __reduce_max_sync(0xffffffffu, mx0);
    mn1 = __reduce_min_sync(0xffffffffu, mn1); mx1 = __reduce_max_sync(0xffffffffu, mx1);
    mn2 = __reduce_min_sync(0xffffffffu, mn2); mx2 = __reduce_max_sync(0xffffffffu, mx2);
    if (tx == 0) {
        atomicMin(&fmin_s[0], mn0); atomicMax(&fmax_s[0], mx0);
        atomicMin(&fmin_s[1], mn1); atomicMax(&fmax_s[1], mx1);
        atomicMin(&fmin_s[2], mn2); atomicMax(&fmax_s[2], mx2);
    }
    __syncthreads();
    // source box [lo, lo + S) per axis covering every stencil of the block
    const int lo1 = i1b + fmin_s[0] - 1;
    const int lo2 = blockIdx.y * T2 + fmin_s[1] - 1;
    const int lo3 = blockIdx.x * T3 + fmin_s[2] - 1;
    const long long S1l = (long long)T1 + 3 + fmax_s[0] - fmin_s[0];
    const long long S2l = (long long)T2 + 3 + fmax_s[1] - fmin_s[1];
    const long long S3l = (long long)T3 + 3 + fmax_s[2] - fmin_s[2];
    const bool use_box = S1l * S2l * S3l <= BOX_CAP;
    const int S2 = (int)S2l, S3 = (int)S3l;
    if (use_box) {
        const int rows = (int)(S1l * S2l);
        for (int r = ty; r < rows; r += T2) {
            const int z = r / S2, y = r - z * S2;
            const int g1 = wrap_index(lo1 + z, d.n1), g2 = wrap_index(lo2 + y, d.n2);
            const float *srow = a.src + ((long long)g1 * d.n2 + g2) * d.n3;
            float *brow = box + r * S3;
            for (int x = tx; x < S3; x += T3) brow[x] = __ldg(srow + wrap_index(lo3 + x, d.n3));
        }
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < T1; ++t) {
        const int i1 = i1b + t;
        if (!(ok23 && i1 < d.n1)) continue;
        const long long id = ((long long)i1 * d.n2 + i2) * d.n3 + i3;
        float val;
        if (use_box) {
            const float fl0 = floorf(dd[t][0]), fl1 = floorf(dd[t][1]), fl2 = floorf(dd[t][2]);
            float w1[4], w2[4], w3[4];
            lagrange4(dd[t][0] - fl0, w1);
            lagrange4(dd[t][1] - fl1, w2);
            lagrange4(dd[t][2] - fl2, w3);
            const int b1 = i1 + (int)fl0 - 1 - lo1;
            const int b2 = i2 + (int)fl1 - 1 - lo2;
            const int b3 = i3 + (int)fl2 - 1 - lo3;
            const float *p = box + (b1 * S2 + b2) * S3 + b3;
            float acc = 0.f;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float s2 = 0.f;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float *q = p + (i * S2 + j) * S3;
                    float s3 = w3[0] * q[0];
                    s3 = fmaf(w3[1], q[1], s3);
                    s3 = fmaf(w3[2], q[2], s3);
                    s3 = fmaf(w3[3], q[3], s3);
                    s2 = fmaf(w2[j], s3, s2);
                }
                acc = fmaf(w1[i], s2, acc);
            }
            val = acc;
        } else {
            Pt p;
            p.i1 = i1; p.i2 = i2; p.i3 = i3;
            val = interp_at(a.src, d, p, dd[t][0], dd[t][1], dd[t][2]);
        }
        if (MODE == SL_PLAIN) {
            a.dst[id] = val;
        } else if (MODE == SL_ADJ) {
            a.dst[id] = a.aux[id] * val;
        } else if (MODE == SL_ADJFAC) {
            const float dx = a.aux[id];
            a.dst[id] = 1.f + 0.5f * a.dt * (val + dx) + 0.5f * a.dt * a.dt * dx * val;
        } else {
            const float f = -(a.vt[id] * a.gm[id] + a.vt[N + id] * a.gm[N + id] +
                              a.vt[2 * N + id] * a.gm[2 * N + id]);
            a.dst[id] = fmaf(a.dt, f, val);
        }
    }
}

// ---------------------------------------------------------------------------
// Lean global-memory gather (one thread per voxel, L1-cached).  A voxel whose
// 4x4x4 stencil does not cross the periodic boundary (most of them) forms one
// base pointer and reads the 64 taps with row offsets plus immediate column
// offsets; the few stencils that wrap take the per-axis wrapped path.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float gather_lean(const float *__restrict__ f, const Dims &d, int i1,
                                             int i2, int i3, float d1, float d2, float d3) {
    const float fl1 = floorf(d1), fl2 = floorf(d2), fl3 = floorf(d3);
    float w1[4], w2[4], w3[4];
    lagrange4(d1 - fl1, w1);
    lagrange4(d2 - fl2, w2);
    lagrange4(d3 - fl3, w3);
    const int b1 = i1 + floor_int(d1) - 1, b2 = i2 + floor_int(d2) - 1, b3 = i3 + floor_int(d3) - 1;
    const int s2 = d.n3, s1 = d.n2 * d.n3;
    if ((unsigned)b1 <= (unsigned)(d.n1 - 4) && (unsigned)b2 <= (unsigned)(d.n2 - 4) &&
        (unsigned)b3 <= (unsigned)(d.n3 - 4)) {
        const float *p = f + ((long long)b1 * d.n2 + b2) * d.n3 + b3;
        float acc = 0.f;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            float sa = 0.f;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const float *q = p + a * s1 + b * s2;
                float s3 = w3[0] * __ldg(q);
                s3 = fmaf(w3[1], __ldg(q + 1), s3);
                s3 = fmaf(w3[2], __ldg(q + 2), s3);
                s3 = fmaf(w3[3], __ldg(q + 3), s3);
                sa = fmaf(w2[b], s3, sa);
            }
            acc = fmaf(w1[a], sa, acc);
        }
        return acc;
    }
    Axis4 a1, a2, a3;
    axis_stencil(i1, d1, d.n1, s1, a1);
    axis_stencil(i2, d2, d.n2, s2, a2);
    axis_stencil(i3, d3, d.n3, 1, a3);
    return gather64(f, a1, a2, a3);
}

template <int MODE>
__global__ void __launch_bounds__(BX * BY)
k_sl_lean(SlArgs a, Dims d) {
    const int i3 = blockIdx.x * BX + threadIdx.x;
    const int i2 = blockIdx.y * BY + threadIdx.y;
    const int i1 = blockIdx.z;
    if (i3 >= d.n3 || i2 >= d.n2) return;
    const long long N = d.N;
    const long long id = ((long long)i1 * d.n2 + i2) * d.n3 + i3;
    const float val = gather_lean(a.src, d, i1, i2, i3, a.disp[id], a.disp[N + id], a.disp[2 * N + id]);
    if (MODE == SL_PLAIN) {
        a.dst[id] = val;
    } else if (MODE == SL_ADJ) {
        a.dst[id] = a.aux[id] * val;
    } else if (MODE == SL_ADJFAC) {
        const float dx = a.aux[id];
        a.dst[id] = 1.f + 0.5f * a.dt * (val + dx) + 0.5f * a.dt * a.dt * dx * val;
    } else {
        const float f = -(a.vt[id] * a.gm[id] + a.vt[N + id] * a.gm[N + id] +
                          a.vt[2 * N + id] * a.gm[2 * N + id]);
        a.dst[id] = fmaf(a.dt, f, val);
    }
}

inline dim3 grid_tiled(const Dims &d) {
    return dim3((d.n3 + T3 - 1) / T3, (d.n2 + T2 - 1) / T2, (d.n1 + T1 - 1) / T1);
}

template <int MODE>
void launch_tiled(const Dims &d, const SlArgs &a, cudaStream_t st) {
    k_sl_lean<MODE><<<dim3((d.n3 + BX - 1) / BX, (d.n2 + BY - 1) / BY, d.n1), dim3(BX, BY), 0, st>>>(a, d);
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
    SlArgs a{f, disp, out, nullptr, nullptr, nullptr, 0.f};
    launch_tiled<SL_PLAIN>(d, a, st);
}

void launch_adjoint_factor(const Dims &d, int nt, const float *divv, const float *dispp,
                           float *cfac, cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_FOOTPOINT, st, 20.0 * d.N);
    SlArgs a{divv, dispp, cfac, divv, nullptr, nullptr, 1.f / nt};
    launch_tiled<SL_ADJFAC>(d, a, st);
}

void launch_state_step(const Dims &d, const float *src, const float *dispm, float *dst,
                       cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_STATE, st, 20.0 * d.N);
    SlArgs a{src, dispm, dst, nullptr, nullptr, nullptr, 0.f};
    launch_tiled<SL_PLAIN>(d, a, st);
}

void launch_adjoint_step(const Dims &d, const float *src, const float *dispp, const float *cfac,
                         float *dst, cudaStream_t st, Profiler *prof, int kclass) {
    ProfScope ps(prof, kclass, st, 24.0 * d.N);
    SlArgs a{src, dispp, dst, cfac, nullptr, nullptr, 0.f};
    launch_tiled<SL_ADJ>(d, a, st);
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
    SlArgs a{src, dispm, dst, nullptr, vt, gm_next, dt};
    launch_tiled<SL_INCSTATE>(d, a, st);
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
