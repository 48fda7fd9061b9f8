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
// The adjoint steps can also carry the body force of Eq. 3.3 / 3.6,
// b = sum_j w_j l^j grad m^j (trapezoid weights w_j), along: each step adds
// its own term to b while l^{j-1} is still in registers, so no later pass
// re-reads the whole trajectories.
// The foot points are stored as displacements in grid-index units, so the
// integer part and the interpolation weight of each axis come from a small
// number (no loss of precision at large grid indices).
//
// The time-step kernels stage the source field in shared-memory halo boxes
// (k_sl_pipe).  The cubic foot points (k_footpoints_box) walk the same tiles
// and stage the three components of v in shared-memory boxes sized by each
// tile's own predictor floor range; the trilinear foot points
// (k_footpoints) gather v from global memory, one thread per voxel.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <type_traits>

#include "claire_internal.cuh"
#include "reduce.cuh"

namespace claire {

namespace {

constexpr int BX = 32, BY = 8;

// Stored fields are FP32 or, in the FP16-storage form, FP16; arithmetic is
// FP32 either way (FP16 values widen on load, results round to nearest even
// on store).
__device__ __forceinline__ float ldf(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ldf(const __half *p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ void stf(float *p, float v) { *p = v; }

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

template <typename T>
__device__ __forceinline__ float gather64(const T *__restrict__ f, const Axis4 &a1,
                                          const Axis4 &a2, const Axis4 &a3) {
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float s2 = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const T *row = f + a1.o[i] + a2.o[j];
            float s3 = a3.w[0] * ldf(row + a3.o[0]);
            s3 = fmaf(a3.w[1], ldf(row + a3.o[1]), s3);
            s3 = fmaf(a3.w[2], ldf(row + a3.o[2]), s3);
            s3 = fmaf(a3.w[3], ldf(row + a3.o[3]), s3);
            s2 = fmaf(a2.w[j], s3, s2);
        }
        acc = fmaf(a1.w[i], s2, acc);
    }
    return acc;
}

// trilinear (first-order Lagrange) periodic interpolation at i + disp
template <typename T>
__device__ __forceinline__ float gather8(const T *__restrict__ f, const Dims &d, int i1, int i2,
                                         int i3, float d1, float d2, float d3) {
    const float fl1 = floorf(d1), fl2 = floorf(d2), fl3 = floorf(d3);
    const float t1 = d1 - fl1, t2 = d2 - fl2, t3 = d3 - fl3;
    const int a0 = wrap_index(i1 + (int)fminf(fmaxf(fl1, -1.0e6f), 1.0e6f), d.n1);
    const int b0 = wrap_index(i2 + (int)fminf(fmaxf(fl2, -1.0e6f), 1.0e6f), d.n2);
    const int c0 = wrap_index(i3 + (int)fminf(fmaxf(fl3, -1.0e6f), 1.0e6f), d.n3);
    const int a1 = a0 + 1 == d.n1 ? 0 : a0 + 1, b1 = b0 + 1 == d.n2 ? 0 : b0 + 1;
    const int c1 = c0 + 1 == d.n3 ? 0 : c0 + 1;
    const long long s1 = (long long)d.n2 * d.n3, s2 = d.n3;
    const T *r00 = f + a0 * s1 + b0 * s2, *r01 = f + a0 * s1 + b1 * s2;
    const T *r10 = f + a1 * s1 + b0 * s2, *r11 = f + a1 * s1 + b1 * s2;
    const float x00 = fmaf(t3, ldf(r00 + c1) - ldf(r00 + c0), ldf(r00 + c0));
    const float x01 = fmaf(t3, ldf(r01 + c1) - ldf(r01 + c0), ldf(r01 + c0));
    const float x10 = fmaf(t3, ldf(r10 + c1) - ldf(r10 + c0), ldf(r10 + c0));
    const float x11 = fmaf(t3, ldf(r11 + c1) - ldf(r11 + c0), ldf(r11 + c0));
    const float y0 = fmaf(t2, x01 - x00, x00), y1 = fmaf(t2, x11 - x10, x10);
    return fmaf(t1, y1 - y0, y0);
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

// ---------------------------------------------------------------------------
// foot points: Heun (RK2) backward (sign -1) and forward (sign +1) in one pass
//   y* = x + s dt v(x);  X = x + s dt/2 (v(x) + v(y*));  disp = (X - x)/h
// ---------------------------------------------------------------------------
__device__ __forceinline__ int floor_int(float x) {
    return (int)fminf(fmaxf(floorf(x), -1.0e6f), 1.0e6f);
}

// One thread per voxel (the trilinear form); the box geometry of its outputs
// comes from k_tile_ranges.
template <int ORDER>
__global__ void __launch_bounds__(BX * BY)
k_footpoints(const float *__restrict__ v, float *__restrict__ dispm, float *__restrict__ dispp,
             Dims d, float dt, float ih1, float ih2, float ih3) {
    const Pt p = this_point(d);
    if (!p.ok) return;
    const long long N = d.N;
    const float v1 = v[p.id], v2 = v[N + p.id], v3 = v[2 * N + p.id];
    // X- (side 0) and X+ (side 1); a side whose output is null is skipped
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        float *out = s == 0 ? dispm : dispp;
        if (!out) continue;
        const float sg = s == 0 ? -1.f : 1.f;
        const float q1 = sg * dt * v1 * ih1, q2 = sg * dt * v2 * ih2, q3 = sg * dt * v3 * ih3;
        float w1, w2, w3;
        if (ORDER == 1) {
            w1 = gather8(v, d, p.i1, p.i2, p.i3, q1, q2, q3);
            w2 = gather8(v + N, d, p.i1, p.i2, p.i3, q1, q2, q3);
            w3 = gather8(v + 2 * N, d, p.i1, p.i2, p.i3, q1, q2, q3);
        } else {
            Axis4 a1, a2, a3;
            axis_stencil(p.i1, q1, d.n1, d.n2 * d.n3, a1);
            axis_stencil(p.i2, q2, d.n2, d.n3, a2);
            axis_stencil(p.i3, q3, d.n3, 1, a3);
            w1 = gather64(v, a1, a2, a3);
            w2 = gather64(v + N, a1, a2, a3);
            w3 = gather64(v + 2 * N, a1, a2, a3);
        }
        const float hs = 0.5f * sg * dt;
        out[p.id] = hs * (v1 + w1) * ih1;
        out[N + p.id] = hs * (v2 + w2) * ih2;
        out[2 * N + p.id] = hs * (v3 + w3) * ih3;
    }
}

// ---------------------------------------------------------------------------
// Arguments shared by the semi-Lagrangian step kernels.
// ---------------------------------------------------------------------------
// SL_INCLAST: the last incremental-state step, whose epilogue writes the
// incremental adjoint's final condition lt(1) = -mt(1) (and mt(1)) directly,
// and optionally the first body-force term w_nt lt(1) grad m(1).
// SL_ADJACC: adjoint step that adds w l^{j-1} grad m^{j-1} to the body force;
// SL_ADJDOT: the same, and the block partials of p . b of the finished sum
// (b . b without p).
enum SlMode { SL_PLAIN = 0, SL_ADJ = 1, SL_INCSTATE = 2, SL_ADJFAC = 3, SL_INCLAST = 4, SL_ADJACC = 5, SL_ADJDOT = 6 };

// TS: storage type of the gathered and written field; TG: of grad m
template <typename TS = float, typename TG = float>
struct SlArgsT {
    const TS *src;      // field gathered at the foot points
    const float *disp;  // foot point minus grid point, index units, [3][N]
    TS *dst;
    const float *aux;   // SL_ADJ: c;  SL_ADJFAC: div v on the grid
    const float *vt;    // SL_INCSTATE: vt [3][N]
    const TG *gm;       // SL_INCSTATE: grad m^{j+1};  SL_ADJACC/SL_ADJDOT: grad m^{j-1}  [3][N]
    float dt;
    __half *dst_h = nullptr;  // SL_PLAIN / SL_ADJ / SL_ADJACC: optional FP16 copy of dst (stored trajectories)
    float *dst2 = nullptr;    // SL_INCLAST: mt(1) (optional)
    float *acc = nullptr;     // body force b [3][N]: SL_ADJACC/SL_ADJDOT update it, SL_INCLAST starts it (optional)
    float w = 0.f;            // SL_ADJACC/SL_ADJDOT: trapezoid weight of the new term (dt, dt/2 at j = 0)
    const float *pv = nullptr;      // SL_ADJDOT: p [3][N] (null: the dot is b . b)
    double *partial = nullptr;      // SL_ADJDOT: one partial sum of p . b per block
};
using SlArgs = SlArgsT<float, float>;


// ---------------------------------------------------------------------------
// Lean global-memory gather (one thread per voxel, L1-cached).  A voxel whose
// 4x4x4 stencil does not cross the periodic boundary (most of them) forms one
// base pointer and reads the 64 taps with row offsets plus immediate column
// offsets; the few stencils that wrap take the per-axis wrapped path.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ float gather_lean(const T *__restrict__ f, const Dims &d, int i1,
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
        const T *p = f + ((long long)b1 * d.n2 + b2) * d.n3 + b3;
        float acc = 0.f;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            float sa = 0.f;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const T *q = p + a * s1 + b * s2;
                float s3 = w3[0] * ldf(q);
                s3 = fmaf(w3[1], ldf(q + 1), s3);
                s3 = fmaf(w3[2], ldf(q + 2), s3);
                s3 = fmaf(w3[3], ldf(q + 3), s3);
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

// ---------------------------------------------------------------------------
// Software-pipelined tiled semi-Lagrangian step (the production path).
// Persistent blocks walk the tiles of 32 x 8 x 4 voxels.  Every tile has a box
// entry (written by the foot-point kernel with the displacements, or by
// k_tile_ranges): the smallest floor of its displacements per axis, which
// fixes where its shared-memory source box starts, and whether the floors
// fit the box.  While a block computes tile k from one shared-memory buffer,
// cp.async already copies the box of tile k+1 into the other.  The
// displacements and epilogue inputs of a tile are loaded when the tile starts,
// not a tile ahead: that holds half the registers (three blocks per SM for the
// incremental state, which has six epilogue inputs a voxel), and the loads
// still overlap the box wait and the other resident blocks (measured at
// 256^3: state 199 -> 182 us, adjoint 205 -> 187 us, incremental state
// 234 -> 207 us, accumulating adjoint 242 -> 230 us).  The 64 taps of
// a voxel are then shared-memory reads with immediate offsets, the same
// instruction stream for every lane (the periodic wrap happened once, when
// the box was fetched).  A tile whose floors span more than the box gathers
// from global memory instead (the decision is uniform per tile), so a region
// of large displacements slows only its own tiles.
// ---------------------------------------------------------------------------
constexpr int PT3 = 32, PT2 = 8, PT1 = 4;
// box geometry, fixed at compile time: floors of a tile's displacements may
// span BOX_SPAN + 1 consecutive integers per axis (per-step displacements that
// vary by about a cell over a tile); wider ranges take the global-memory gather
constexpr int BOX_SPAN = 2;
constexpr int BS1 = PT1 + 3 + BOX_SPAN, BS2 = PT2 + 3 + BOX_SPAN, BS3 = PT3 + 3 + BOX_SPAN;
constexpr int BOX_PITCH = 64;  // floats per box row: rows start on bank 0
constexpr int BOX_FLOATS = BS1 * BS2 * BOX_PITCH;
static_assert(BS3 <= BOX_PITCH && BS3 > PT3, "box row must fit one pitch and exceed a warp");

// Debug build (-DCLAIRE_CHECKS): every box stencil origin is checked before
// its 64 taps are read -- inside the buffer and inside the columns the box
// copy wrote -- and a violation is counted in g_check_count and its taps are
// not read (the value becomes 0).  The release build compiles the check away.
// The host model of the same geometry is tests/test_box_geometry.py.
#ifdef CLAIRE_CHECKS
__device__ unsigned long long g_check_count;
__device__ __forceinline__ bool box_origin_ok(int b1, int b2, int b3, int ncols) {
    const bool ok = b1 >= 0 && b1 + 3 < BS1 && b2 >= 0 && b2 + 3 < BS2 && b3 >= 0 && b3 + 3 < ncols;
    if (!ok) atomicAdd(&g_check_count, 1ull);
    return ok;
}
#else
__device__ __forceinline__ bool box_origin_ok(int, int, int, int) { return true; }
#endif

__device__ __forceinline__ void cp_async4(float *smem, const float *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int NPEND>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(NPEND) : "memory");
}

// epilogue inputs prefetched with the next tile's displacements
template <int MODE> struct EpiCount {
    static constexpr int v = (MODE == SL_INCSTATE || MODE == SL_INCLAST) ? 6 : (MODE == SL_PLAIN ? 0 : 1);
};
// epilogue inputs of the accumulating adjoint steps, loaded when a tile
// starts (grad m^{j-1}, b, and p for the dot): prefetching them a tile ahead
// as well would hold twice as many registers
template <int MODE> struct EarlyCount {
    static constexpr int v = MODE == SL_ADJACC ? 6 : (MODE == SL_ADJDOT ? 9 : 0);
};

template <int MODE, typename A>
__device__ __forceinline__ void sl_load_early(const A &a, long long id, long long N, float *x) {
    if (MODE == SL_ADJACC || MODE == SL_ADJDOT) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            x[k] = ldf(a.gm + k * N + id);
            x[3 + k] = a.acc[k * N + id];
            if (MODE == SL_ADJDOT) x[6 + k] = a.pv ? a.pv[k * N + id] : 0.f;
        }
    }
}

template <int MODE, typename A>
__device__ __forceinline__ void sl_epilogue(const A &a, long long id, long long N, float val, const float *e,
                                            const float *x, Acc2 &dot) {
    if (MODE == SL_PLAIN) {
        stf(a.dst + id, val);
        if (a.dst_h) a.dst_h[id] = __float2half_rn(val);
    } else if (MODE == SL_ADJ) {
        const float r = e[0] * val;
        stf(a.dst + id, r);
        if (a.dst_h) a.dst_h[id] = __float2half_rn(r);
    } else if (MODE == SL_ADJFAC) {
        const float dx = e[0];
        stf(a.dst + id, 1.f + 0.5f * a.dt * (val + dx) + 0.5f * a.dt * a.dt * dx * val);
    } else if (MODE == SL_INCSTATE) {
        const float f = -(e[0] * e[3] + e[1] * e[4] + e[2] * e[5]);
        stf(a.dst + id, fmaf(a.dt, f, val));
    } else if (MODE == SL_INCLAST) {
        // u(1) = u^{nt-1}(X-) + dt f(1); mt(1) = u(1) - dt/2 f(1); lt(1) = -mt(1)
        const float f = -(e[0] * e[3] + e[1] * e[4] + e[2] * e[5]);
        const float m = fmaf(a.dt, f, val) - 0.5f * a.dt * f;
        stf(a.dst + id, -m);
        if (a.dst2) a.dst2[id] = m;
        if (a.acc) {
            const float l = (0.5f * a.dt) * (-m);
#pragma unroll
            for (int k = 0; k < 3; ++k) a.acc[k * N + id] = l * e[3 + k];
        }
    } else if (MODE == SL_ADJACC || MODE == SL_ADJDOT) {
        const float r = e[0] * val;
        stf(a.dst + id, r);
        if (a.dst_h) a.dst_h[id] = __float2half_rn(r);
        const float l = a.w * r;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float b = fmaf(l, x[k], x[3 + k]);
            a.acc[k * N + id] = b;
            if (MODE == SL_ADJDOT) dot.add_prod(a.pv ? x[6 + k] : b, b);
        }
    }
}

template <int MODE, typename A>
__device__ __forceinline__ void sl_load_epi(const A &a, long long id, long long N, float *e) {
    if (MODE == SL_ADJ || MODE == SL_ADJFAC || MODE == SL_ADJACC || MODE == SL_ADJDOT) {
        e[0] = a.aux[id];
    } else if (MODE == SL_INCSTATE || MODE == SL_INCLAST) {
        e[0] = a.vt[id]; e[1] = a.vt[N + id]; e[2] = a.vt[2 * N + id];
        e[3] = ldf(a.gm + id); e[4] = ldf(a.gm + N + id); e[5] = ldf(a.gm + 2 * N + id);
    }
}

// Box copy of tile rows [lo1, lo1 + BS1) x [lo2, lo2 + BS2) x [lo3, lo3 + BS3)
// of a periodic field.  Chunked (n3 a multiple of 4 and a 16-byte aligned
// field): 16-byte cp.async of 40 floats per row from lo3 rounded down to a
// multiple of 4, three rows per warp instruction; the stencil columns then sit
// box_shift() floats further right.  Otherwise one float per lane and column.
constexpr int BOX_CH = 10;  // 16-byte chunks per box row
constexpr int BOX_ROWS = BS1 * BS2;
static_assert(4 * BOX_CH >= BS3 + 3 && 4 * BOX_CH <= BOX_PITCH, "chunked box row must cover the shifted row");

__device__ __forceinline__ void cp_async16(float *smem, const float *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

__device__ __forceinline__ int box_shift(int lo3, bool chunked) { return chunked ? lo3 - (lo3 & ~3) : 0; }
// columns of a box row that the copy writes
__device__ __forceinline__ int box_cols(bool chunked) { return chunked ? 4 * BOX_CH : BS3; }

__device__ __forceinline__ void box_copy(const float *__restrict__ src, const Dims &d, long long plane, int lo1,
                                         int lo2, int lo3, float *buf, bool chunked) {
    const int tx = threadIdx.x, ty = threadIdx.y;
    if (chunked) {
        const int lrow = tx / BOX_CH, lch = tx - lrow * BOX_CH;
        if (tx < 3 * BOX_CH) {
            const int gx = wrap_index((lo3 & ~3) + 4 * lch, d.n3);
#pragma unroll
            for (int i = 0; i < (BOX_ROWS + 3 * PT2 - 1) / (3 * PT2); ++i) {
                const int row = 3 * (ty + PT2 * i) + lrow;
                if (row < BOX_ROWS) {
                    const int z = row / BS2, y = row - z * BS2;
                    cp_async16(buf + row * BOX_PITCH + 4 * lch,
                               src + wrap_index(lo1 + z, d.n1) * plane + (long long)wrap_index(lo2 + y, d.n2) * d.n3 + gx);
                }
            }
        }
    } else {
        const int xa = wrap_index(lo3 + tx, d.n3);
        const bool two = tx < BS3 - PT3;
        const int xb = wrap_index(lo3 + tx + PT3, d.n3);
#pragma unroll
        for (int yy = 0; yy < (BS2 + PT2 - 1) / PT2; ++yy) {
            const int y = ty + yy * PT2;
            if (y < BS2) {
                const long long g2 = (long long)wrap_index(lo2 + y, d.n2) * d.n3;
#pragma unroll
                for (int z = 0; z < BS1; ++z) {
                    const float *srow = src + wrap_index(lo1 + z, d.n1) * plane + g2;
                    float *brow = buf + (z * BS2 + y) * BOX_PITCH;
                    cp_async4(brow + tx, srow + xa);
                    if (two) cp_async4(brow + tx + PT3, srow + xb);
                }
            }
        }
    }
    cp_async_commit();
}

// 64-tap tricubic sum from a box position; pairs of rows go through the
// paired FP32 instructions (FMUL2/FFMA2), the x2 and x1 contractions too
__device__ __forceinline__ float box_cubic(const float *p, const float w1[4], const float w2[4], const float w3[4]) {
    const float2 c0 = make_float2(w3[0], w3[0]), c1 = make_float2(w3[1], w3[1]);
    const float2 c2 = make_float2(w3[2], w3[2]), c3 = make_float2(w3[3], w3[3]);
    const float2 w2a = make_float2(w2[0], w2[1]), w2b = make_float2(w2[2], w2[3]);
    float2 u = make_float2(0.f, 0.f);
#pragma unroll
    for (int ia = 0; ia < 4; ++ia) {
        float2 sr[2];
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const float *q0 = p + (ia * BS2 + 2 * m) * BOX_PITCH, *q1 = q0 + BOX_PITCH;
            float2 t = __fmul2_rn(c0, make_float2(q0[0], q1[0]));
            t = __ffma2_rn(c1, make_float2(q0[1], q1[1]), t);
            t = __ffma2_rn(c2, make_float2(q0[2], q1[2]), t);
            t = __ffma2_rn(c3, make_float2(q0[3], q1[3]), t);
            sr[m] = t;
        }
        const float2 tr = __ffma2_rn(sr[1], w2b, __fmul2_rn(sr[0], w2a));
        const float2 wa = make_float2(w1[ia], w1[ia]);
        u = ia == 0 ? __fmul2_rn(tr, wa) : __ffma2_rn(tr, wa, u);
    }
    return u.x + u.y;
}

// trilinear sum from the cubic stencil origin p (nodes floor and floor + 1)
__device__ __forceinline__ float box_linear(const float *p, float u1, float u2, float u3) {
    p += (BS2 + 1) * BOX_PITCH + 1;
    const float x00 = fmaf(u3, p[1] - p[0], p[0]);
    const float x01 = fmaf(u3, p[BOX_PITCH + 1] - p[BOX_PITCH], p[BOX_PITCH]);
    const float *p1 = p + BS2 * BOX_PITCH;
    const float x10 = fmaf(u3, p1[1] - p1[0], p1[0]);
    const float x11 = fmaf(u3, p1[BOX_PITCH + 1] - p1[BOX_PITCH], p1[BOX_PITCH]);
    const float y0 = fmaf(u2, x01 - x00, x00), y1 = fmaf(u2, x11 - x10, x10);
    return fmaf(u1, y1 - y0, y0);
}

// resident blocks per SM (launch bounds and grid size): the accumulating
// adjoint steps hold nine or twelve inputs a voxel and keep two
template <int MODE> struct SlOcc {
    static constexpr int v = (MODE == SL_ADJACC || MODE == SL_ADJDOT) ? 2 : 3;
};

// tiles of block b: a contiguous range, so neighbouring tiles (which share
// halo rows in L2) run on the same block one after the other
__device__ __forceinline__ void tile_range(int ntiles, int &tbeg, int &tend) {
    tbeg = (int)((long long)blockIdx.x * ntiles / gridDim.x);
    tend = (int)((long long)(blockIdx.x + 1) * ntiles / gridDim.x);
}

// floors inside the clamp of floor_int: a non-finite or huge displacement
// (clamped to +-1e6 there, while the box path converts floorf directly) sends
// the tile to the gather path, whose stencil clamps
__device__ __forceinline__ bool floor_sane(int lo, int hi) { return lo > -1000000 && hi < 1000000; }

// Box entry of one tile of a displacement field: {lo1, lo2, lo3, ok}, lo_d =
// the smallest floor of the tile's displacements along axis d; ok = 1 when on
// every axis the floors span at most BOX_SPAN + 1 consecutive integers (the
// tile's stencils then lie inside the box at lo - 1), 0 otherwise (the tile
// gathers from global memory).  lo, hi: this thread's per-axis floor min and
// max over its voxels of the tile; red: [PT2][6] shared ints.  Contains one
// barrier; the entry is written by thread (0, 0) after a second pass over red,
// so the caller needs a barrier before red is written again.
__device__ __forceinline__ void tile_box_reduce(const int lo[3], const int hi[3], int (*red)[6], int4 *out) {
    const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int a = __reduce_min_sync(0xffffffffu, lo[c]), b = __reduce_max_sync(0xffffffffu, hi[c]);
        if (tx == 0) {
            red[ty][2 * c] = a;
            red[ty][2 * c + 1] = b;
        }
    }
    __syncthreads();
    if (ty == 0) {
        int x = 0;
        if (tx < 6) {
            x = red[0][tx];
            for (int y = 1; y < PT2; ++y) x = (tx & 1) ? max(x, red[y][tx]) : min(x, red[y][tx]);
        }
        const int l0 = __shfl_sync(0xffffffffu, x, 0), h0 = __shfl_sync(0xffffffffu, x, 1);
        const int l1 = __shfl_sync(0xffffffffu, x, 2), h1 = __shfl_sync(0xffffffffu, x, 3);
        const int l2 = __shfl_sync(0xffffffffu, x, 4), h2 = __shfl_sync(0xffffffffu, x, 5);
        if (tx == 0) {
            const bool ok = h0 - l0 <= BOX_SPAN && h1 - l1 <= BOX_SPAN && h2 - l2 <= BOX_SPAN && floor_sane(l0, h0) &&
                            floor_sane(l1, h1) && floor_sane(l2, h2);
            *out = make_int4(l0, l1, l2, ok ? 1 : 0);
        }
    }
}

// block partial of the dot product of the accumulating adjoint step
template <int MODE>
__device__ __forceinline__ void sl_dot_store(const Acc2 &dot, double *partial) {
    if (MODE == SL_ADJDOT) {
        const double s = block_sum_n<PT3 * PT2>(dot.value(), threadIdx.y * PT3 + threadIdx.x);
        if (threadIdx.x == 0 && threadIdx.y == 0) partial[blockIdx.x] = s;
    }
}

// One tile of a step by global-memory gathers, for tiles whose displacement
// floors span more than the box holds.  It loads the tile's inputs itself and
// returns its part of the epilogue's dot product.  Not inlined, and called
// outside the box path's voxel loop, so that its registers and call frame
// stay out of the box path.
template <int MODE, int ORDER, typename TS, typename TG>
__device__ __noinline__ Acc2 sl_gather_tile(const SlArgsT<TS, TG> &a, const Dims &d, int t1, int t2, int t3) {
    constexpr int NE = EpiCount<MODE>::v > 0 ? EpiCount<MODE>::v : 1;
    constexpr int NX = EarlyCount<MODE>::v > 0 ? EarlyCount<MODE>::v : 1;
    Acc2 dot;
    const int i3 = t3 * PT3 + threadIdx.x, i2 = t2 * PT2 + threadIdx.y;
    if (i3 >= d.n3 || i2 >= d.n2) return dot;
    const long long N = d.N, plane = (long long)d.n2 * d.n3;
    for (int t = 0; t < PT1; ++t) {
        const int i1 = t1 * PT1 + t;
        if (i1 >= d.n1) break;
        const long long id = i1 * plane + (long long)i2 * d.n3 + i3;
        const float d1 = a.disp[id], d2 = a.disp[N + id], d3 = a.disp[2 * N + id];
        const float val = ORDER == 1 ? gather8(a.src, d, i1, i2, i3, d1, d2, d3)
                                     : gather_lean(a.src, d, i1, i2, i3, d1, d2, d3);
        float e[NE], x[NX];
        sl_load_epi<MODE>(a, id, N, e);
        sl_load_early<MODE>(a, id, N, x);
        sl_epilogue<MODE>(a, id, N, val, e, x, dot);
    }
    return dot;
}

constexpr int GTAB = 64;  // box entries a block stages in shared memory at a time

// FULL: the grid is a whole number of tiles on every axis, so no voxel of a
// tile needs a bounds check (measured ~5% of the step time at 256^3)
template <int MODE, int ORDER, typename TS = float, typename TG = float, bool FULL = false>
__global__ void __launch_bounds__(PT3 * PT2, SlOcc<MODE>::v)
k_sl_pipe(SlArgsT<TS, TG> a, Dims d, const int4 *__restrict__ tiles, int chunked_in) {
    static_assert(std::is_same<TS, float>::value, "the box path stages FP32 source fields");
    constexpr int NE = EpiCount<MODE>::v > 0 ? EpiCount<MODE>::v : 1;
    constexpr int NX = EarlyCount<MODE>::v > 0 ? EarlyCount<MODE>::v : 1;
    Acc2 dot;
    extern __shared__ float smem[];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const bool chunked = chunked_in != 0;
    const int nb3 = (d.n3 + PT3 - 1) / PT3, nb2 = (d.n2 + PT2 - 1) / PT2, nb1 = (d.n1 + PT1 - 1) / PT1;
    const int ntiles = nb3 * nb2 * nb1;
    const long long N = d.N, plane = (long long)d.n2 * d.n3;
    int tbeg, tend;
    tile_range(ntiles, tbeg, tend);
    if (tbeg < tend) {
        // box of a tile at its own floor range g (lo1, lo2, lo3); a tile whose
        // range does not fit (g.w == 0) copies nothing, but still commits a
        // (empty) group so that the wait counts stay the same
        auto issue_box = [&](int t1, int t2, int t3, const int4 &g, float *buf) {
            if (g.w) box_copy(a.src, d, plane, t1 * PT1 + g.x - 1, t2 * PT2 + g.y - 1, t3 * PT3 + g.z - 1, buf, chunked);
            else cp_async_commit();
        };
        // displacements and epilogue inputs of the voxels of a tile
        auto load_regs = [&](int t1, int t2, int t3, float *dd, float *ee) {
            const int i3 = t3 * PT3 + tx, i2 = t2 * PT2 + ty;
            const long long id0 = (long long)t1 * PT1 * plane + (long long)i2 * d.n3 + i3;
#pragma unroll
            for (int t = 0; t < PT1; ++t) {
                if (FULL || (i3 < d.n3 && i2 < d.n2 && t1 * PT1 + t < d.n1)) {
                    const long long id = id0 + t * plane;
                    dd[3 * t] = a.disp[id];
                    dd[3 * t + 1] = a.disp[N + id];
                    dd[3 * t + 2] = a.disp[2 * N + id];
                    sl_load_epi<MODE>(a, id, N, ee + NE * t);
                }
            }
        };

        // the block's box entries are staged in shared memory, GTAB at a time
        // (a register copy of a pending global load would stall each tile)
        __shared__ int4 gtab[GTAB];
        auto stage_entries = [&](int first) {
            for (int k = ty * PT3 + tx; k < GTAB && first + k < tend; k += PT3 * PT2) gtab[k] = tiles[first + k];
        };
        int gbase = tbeg;
        stage_entries(gbase);
        __syncthreads();
        // tile counters of the next tile to fetch (x3 fastest)
        int c3 = tbeg % nb3, c2 = (tbeg / nb3) % nb2, c1 = tbeg / (nb3 * nb2);
        int4 g_cur = gtab[0];
        issue_box(c1, c2, c3, g_cur, smem);
        int cur = 0;
        for (int tile = tbeg; tile < tend; ++tile) {
            const int t1 = c1, t2 = c2, t3 = c3;
            if (++c3 == nb3) {
                c3 = 0;
                if (++c2 == nb2) { c2 = 0; ++c1; }
            }
            // this tile's inputs, loaded now: they arrive while the box of
            // the next tile is issued and this tile's box is awaited
            float cd[PT1 * 3], ce[PT1 * NE], cx[PT1][NX];
            load_regs(t1, t2, t3, cd, ce);
            const int i3 = t3 * PT3 + tx, i2 = t2 * PT2 + ty;
            const long long id0 = (long long)t1 * PT1 * plane + (long long)i2 * d.n3 + i3;
            const bool inplane = FULL || (i3 < d.n3 && i2 < d.n2);
            if (EarlyCount<MODE>::v > 0 && inplane) {
#pragma unroll
                for (int t = 0; t < PT1; ++t)
                    if (FULL || t1 * PT1 + t < d.n1) sl_load_early<MODE>(a, id0 + t * plane, N, cx[t]);
            }
            // entry of the next tile (the table is refilled behind the barrier
            // that follows this tile when the next tile starts a new batch)
            const int4 g_next = tile + 1 < tend && tile + 1 - gbase < GTAB ? gtab[tile + 1 - gbase] : g_cur;
            const bool refill = tile + 1 < tend && tile + 1 - gbase == GTAB;
            if (tile + 1 < tend) {
                if (refill) {
                    // the next batch of entries: its first one is read here
                    // from global memory, the rest after the end barrier
                    const int4 gn = tiles[tile + 1];
                    issue_box(c1, c2, c3, gn, smem + (cur ^ 1) * BOX_FLOATS);
                } else {
                    issue_box(c1, c2, c3, g_next, smem + (cur ^ 1) * BOX_FLOATS);
                }
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
            const float *bx = smem + cur * BOX_FLOATS;
            const int fmn0 = g_cur.x, fmn1 = g_cur.y, fmn2 = g_cur.z;
            const int sh = box_shift(t3 * PT3 + fmn2 - 1, chunked);
            if (!g_cur.w) {
                const Acc2 td = sl_gather_tile<MODE, ORDER>(a, d, t1, t2, t3);
                if (MODE == SL_ADJDOT) dot.add(td.s, td.c);
            } else if (inplane) {
#pragma unroll
                for (int t = 0; t < PT1; ++t) {
                    if (FULL || t1 * PT1 + t < d.n1) {
                        const float *dt3 = cd + 3 * t;
                        const float fl0 = floorf(dt3[0]), fl1 = floorf(dt3[1]), fl2 = floorf(dt3[2]);
                        // stencil origin inside the box; every tap is an immediate offset
                        const int b1 = t + (int)fl0 - fmn0, b2 = ty + (int)fl1 - fmn1, b3 = tx + (int)fl2 - fmn2 + sh;
                        const float *p = bx + (b1 * BS2 + b2) * BOX_PITCH + b3;
                        float acc = 0.f;
                        if (!box_origin_ok(b1, b2, b3, box_cols(chunked))) {
                        } else if (ORDER == 1) {
                            acc = box_linear(p, dt3[0] - fl0, dt3[1] - fl1, dt3[2] - fl2);
                        } else {
                            float w1[4], w2[4], w3[4];
                            lagrange4(dt3[0] - fl0, w1);
                            lagrange4(dt3[1] - fl1, w2);
                            lagrange4(dt3[2] - fl2, w3);
                            acc = box_cubic(p, w1, w2, w3);
                        }
                        sl_epilogue<MODE>(a, id0 + t * plane, N, acc, ce + NE * t, cx[t], dot);
                    }
                }
            }
            __syncthreads();
            cur ^= 1;
            if (refill) {
                gbase = tile + 1;
                stage_entries(gbase);
                __syncthreads();
            }
            g_cur = gtab[tile + 1 - gbase < GTAB ? tile + 1 - gbase : 0];
        }
    }
    sl_dot_store<MODE>(dot, a.partial);
}

// Box entries of every tile of a displacement field (for fields that do not
// come from the foot-point kernel, which writes them itself): persistent
// blocks over the tiles, 12 bytes read per voxel.
__global__ void __launch_bounds__(PT3 * PT2)
k_tile_ranges(const float *__restrict__ disp, Dims d, int4 *__restrict__ tiles) {
    __shared__ int red[PT2][6];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int nb3 = (d.n3 + PT3 - 1) / PT3, nb2 = (d.n2 + PT2 - 1) / PT2, nb1 = (d.n1 + PT1 - 1) / PT1;
    const long long N = d.N, plane = (long long)d.n2 * d.n3;
    int tbeg, tend;
    tile_range(nb3 * nb2 * nb1, tbeg, tend);
    for (int tile = tbeg; tile < tend; ++tile) {
        const int t3 = tile % nb3, r = tile / nb3, t2 = r % nb2, t1 = r / nb2;
        const int i3 = t3 * PT3 + tx, i2 = t2 * PT2 + ty;
        int lo[3] = {0x7fffffff, 0x7fffffff, 0x7fffffff}, hi[3] = {-0x7fffffff, -0x7fffffff, -0x7fffffff};
        if (i3 < d.n3 && i2 < d.n2) {
            for (int t = 0; t < PT1 && t1 * PT1 + t < d.n1; ++t) {
                const long long id = (long long)(t1 * PT1 + t) * plane + (long long)i2 * d.n3 + i3;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int f = floor_int(disp[c * N + id]);
                    lo[c] = min(lo[c], f);
                    hi[c] = max(hi[c], f);
                }
            }
        }
        tile_box_reduce(lo, hi, red, tiles + tile);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Foot points from shared-memory boxes (cubic interpolation of v at the RK2
// predictor).  Persistent blocks walk the 32 x 8 x 4 tiles of the SL steps.
// For each side the block reduces the floor range of its own predictor
// displacements s dt v(x)/h over the tile, copies the three components of v
// over that box into shared memory, and sums the 64 taps of all three
// components with one set of weights: one shared-memory wavefront per tap and
// warp, where the global-memory gather of a misaligned 32-float row costs two
// L1 wavefronts.  A tile whose predictor floors span more than the box allows
// gathers from global memory instead (the decision is uniform per block).
// The block also reduces, per tile and side, the floor range of what it wrote:
// the box entry of that tile for the SL steps.
// ---------------------------------------------------------------------------
constexpr int FP_OCC = 2;  // resident blocks per SM: three component boxes each

// v at the predictor point i + q by global-memory gathers (tiles whose
// predictor floors span more than the box).  Not inlined: its registers stay
// out of the box path's allocation.
__device__ __noinline__ float3 fp_gather3(const float *__restrict__ v, const Dims &d, int i1, int i2, int i3,
                                          float q1, float q2, float q3) {
    Axis4 a1, a2, a3;
    axis_stencil(i1, q1, d.n1, d.n2 * d.n3, a1);
    axis_stencil(i2, q2, d.n2, d.n3, a2);
    axis_stencil(i3, q3, d.n3, 1, a3);
    return make_float3(gather64(v, a1, a2, a3), gather64(v + d.N, a1, a2, a3), gather64(v + 2 * d.N, a1, a2, a3));
}

__global__ void __launch_bounds__(PT3 * PT2, FP_OCC)
k_footpoints_box(const float *__restrict__ v, float *__restrict__ dispm, float *__restrict__ dispp, Dims d,
                 float dt, float ih1, float ih2, float ih3, int chunked_in, int4 *__restrict__ tiles_m,
                 int4 *__restrict__ tiles_p) {
    extern __shared__ float smem[];
    __shared__ int red[PT2][6];
    __shared__ int ored[PT2][6];
    __shared__ int rng[6];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const bool chunked = chunked_in != 0;
    const int nb3 = (d.n3 + PT3 - 1) / PT3, nb2 = (d.n2 + PT2 - 1) / PT2, nb1 = (d.n1 + PT1 - 1) / PT1;
    const long long N = d.N, plane = (long long)d.n2 * d.n3;
    const float ih[3] = {ih1, ih2, ih3};
    int tbeg, tend;
    tile_range(nb3 * nb2 * nb1, tbeg, tend);
    for (int tile = tbeg; tile < tend; ++tile) {
        const int t3 = tile % nb3, r = tile / nb3, t2 = r % nb2, t1 = r / nb2;
        const int i3 = t3 * PT3 + tx, i2 = t2 * PT2 + ty;
        const long long id0 = (long long)t1 * PT1 * plane + (long long)i2 * d.n3 + i3;
        bool ok[PT1];
        float vx[PT1][3];
#pragma unroll
        for (int t = 0; t < PT1; ++t) {
            ok[t] = i3 < d.n3 && i2 < d.n2 && t1 * PT1 + t < d.n1;
#pragma unroll
            for (int c = 0; c < 3; ++c) vx[t][c] = ok[t] ? v[c * N + id0 + t * plane] : 0.f;
        }
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            float *out = s == 0 ? dispm : dispp;
            if (!out) continue;
            const float sdt = s == 0 ? -dt : dt, hs = 0.5f * sdt;
            // floor range of the predictor displacements over the tile
            int lo[3] = {0x7fffffff, 0x7fffffff, 0x7fffffff}, hi[3] = {-0x7fffffff, -0x7fffffff, -0x7fffffff};
#pragma unroll
            for (int t = 0; t < PT1; ++t) {
                if (ok[t]) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const int f = floor_int(sdt * vx[t][c] * ih[c]);
                        lo[c] = min(lo[c], f);
                        hi[c] = max(hi[c], f);
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int a = __reduce_min_sync(0xffffffffu, lo[c]), b = __reduce_max_sync(0xffffffffu, hi[c]);
                if (tx == 0) {
                    red[ty][2 * c] = a;
                    red[ty][2 * c + 1] = b;
                }
            }
            __syncthreads();
            if (ty == 0 && tx < 6) {
                int x = red[0][tx];
                for (int y = 1; y < PT2; ++y) x = (tx & 1) ? max(x, red[y][tx]) : min(x, red[y][tx]);
                rng[tx] = x;
            }
            __syncthreads();
            const int f0 = rng[0], f1 = rng[2], f2 = rng[4];
            const bool fits = rng[1] - f0 <= BOX_SPAN && rng[3] - f1 <= BOX_SPAN && rng[5] - f2 <= BOX_SPAN &&
                              floor_sane(f0, rng[1]) && floor_sane(f1, rng[3]) && floor_sane(f2, rng[5]);
            if (fits) {
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    box_copy(v + c * N, d, plane, t1 * PT1 + f0 - 1, t2 * PT2 + f1 - 1, t3 * PT3 + f2 - 1,
                             smem + c * BOX_FLOATS, chunked);
                cp_async_wait<0>();
                __syncthreads();
            }
            const int sh = box_shift(t3 * PT3 + f2 - 1, chunked);
            // floor range of this side's output over the tile: the box entry
            // of the SL steps that use it
            int omn[3] = {0x7fffffff, 0x7fffffff, 0x7fffffff}, omx[3] = {-0x7fffffff, -0x7fffffff, -0x7fffffff};
#pragma unroll
            for (int t = 0; t < PT1; ++t) {
                if (!ok[t]) continue;
                const float q1 = sdt * vx[t][0] * ih1, q2 = sdt * vx[t][1] * ih2, q3 = sdt * vx[t][2] * ih3;
                float w[3];
                if (fits) {
                    const float fl1 = floorf(q1), fl2 = floorf(q2), fl3 = floorf(q3);
                    const int b1 = t + (int)fl1 - f0, b2 = ty + (int)fl2 - f1, b3 = tx + (int)fl3 - f2 + sh;
                    const float *p = smem + (b1 * BS2 + b2) * BOX_PITCH + b3;
                    float w1[4], w2[4], w3[4];
                    lagrange4(q1 - fl1, w1);
                    lagrange4(q2 - fl2, w2);
                    lagrange4(q3 - fl3, w3);
                    if (box_origin_ok(b1, b2, b3, box_cols(chunked))) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) w[c] = box_cubic(p + c * BOX_FLOATS, w1, w2, w3);
                    } else {
                        w[0] = w[1] = w[2] = 0.f;
                    }
                } else {
                    const float3 g = fp_gather3(v, d, t1 * PT1 + t, i2, i3, q1, q2, q3);
                    w[0] = g.x;
                    w[1] = g.y;
                    w[2] = g.z;
                }
                const long long id = id0 + t * plane;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float o = hs * (vx[t][c] + w[c]) * ih[c];
                    out[c * N + id] = o;
                    const int f = floor_int(o);
                    omn[c] = min(omn[c], f);
                    omx[c] = max(omx[c], f);
                }
            }
            // the boxes, rng and ored are rewritten by the next side or tile
            // only after further barriers, which the first warp reaches after
            // it has read ored
            tile_box_reduce(omn, omx, ored, (s == 0 ? tiles_m : tiles_p) + tile);
            __syncthreads();
        }
    }
}

// SM count of the device current at the first call (thread-safe initialisation)
int num_sms() {
    static const int n = [] {
        int dev = 0, c = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c <= 0) c = 152;
        return c;
    }();
    return n;
}

// 16-byte box rows need rows of a whole number of chunks (4 floats or 8
// halves) and a 16-byte aligned field
template <typename T>
inline int chunk_ok(const Dims &d, const T *f) {
    const int per = 16 / (int)sizeof(T);
    return (d.n3 % per == 0 && ((uintptr_t)f & 15) == 0) ? 1 : 0;
}

inline int pipe_blocks(const Dims &d, int per_sm) {
    const long long ntiles = (long long)((d.n3 + PT3 - 1) / PT3) * ((d.n2 + PT2 - 1) / PT2) *
                             ((d.n1 + PT1 - 1) / PT1);
    // at most kReduceBlocks: a dot-product step leaves one partial sum per block
    long long want = (long long)per_sm * num_sms();
    if (want > kReduceBlocks) want = kReduceBlocks;
    return (int)(ntiles < want ? ntiles : want);
}

// returns the number of blocks launched (the partial sums a dot-product step
// leaves for its finalize)
template <int MODE, int ORDER, typename TS, typename TG, bool FULL>
int launch_pipe_f(const Dims &d, const SlArgsT<TS, TG> &a, const int4 *tiles, cudaStream_t st) {
    const size_t smem = 2 * BOX_FLOATS * sizeof(float);
    // the shared-memory limit is set once per instantiation and device
    static SmemAttr attr;
    attr.ensure(k_sl_pipe<MODE, ORDER, TS, TG, FULL>, (int)smem, "k_sl_pipe");
    const int grid = pipe_blocks(d, SlOcc<MODE>::v);
    k_sl_pipe<MODE, ORDER, TS, TG, FULL><<<grid, dim3(PT3, PT2), smem, st>>>(a, d, tiles, chunk_ok(d, a.src));
    return grid;
}

// kernels one SL step launches
constexpr int kSlLaunches = 1;

inline bool full_tiles(const Dims &d) { return d.n3 % PT3 == 0 && d.n2 % PT2 == 0 && d.n1 % PT1 == 0; }

// the full-tile form for grids of whole tiles, cubic and trilinear (with 8
// taps a voxel the trilinear steps lose relatively more to the bounds checks:
// incremental state 13.8 -> 10.4 ms per 256^3 solve)
template <int MODE, int ORDER, typename TS, typename TG>
int launch_pipe_o(const Dims &d, const SlArgsT<TS, TG> &a, const int4 *tiles, cudaStream_t st) {
    if constexpr (ORDER == 3 || ORDER == 1) {
        if (full_tiles(d)) return launch_pipe_f<MODE, ORDER, TS, TG, true>(d, a, tiles, st);
    }
    return launch_pipe_f<MODE, ORDER, TS, TG, false>(d, a, tiles, st);
}

template <int MODE, typename TS, typename TG>
int launch_pipe(const Dims &d, const SlArgsT<TS, TG> &a, const int4 *tiles, cudaStream_t st) {
    if (d.iorder == 1) return launch_pipe_o<MODE, 1>(d, a, tiles, st);
    return launch_pipe_o<MODE, 3>(d, a, tiles, st);
}

// ----------------------------------------------------------- pointwise ----
constexpr int PT = 256;

template <typename TG>
__global__ void k_incstate_init(const float *__restrict__ vt, const TG *__restrict__ gm,
                                float *__restrict__ u0, long long N, float hdt) {
    for (long long i = blockIdx.x * (long long)PT + threadIdx.x; i < N; i += (long long)gridDim.x * PT) {
        const float f = -(vt[i] * ldf(gm + i) + vt[N + i] * ldf(gm + N + i) + vt[2 * N + i] * ldf(gm + 2 * N + i));
        u0[i] = hdt * f;
    }
}

// the adjoint's final condition (Eq. 3.2) and the first term of the body
// force, with the gradient started at beta A v:
//   l = m1 - m(1),  g = Av + w l grad m(1)   (w = dt/2, trapezoid end point)
template <typename TG>
__global__ void k_adjfinal_acc(const float *__restrict__ m1, const float *__restrict__ m, float *__restrict__ l,
                               __half *__restrict__ l_h, const TG *__restrict__ gm, const float *__restrict__ Av,
                               float *__restrict__ g, float w, long long N) {
    for (long long i = blockIdx.x * (long long)PT + threadIdx.x; i < N; i += (long long)gridDim.x * PT) {
        const float li = m1[i] - m[i];
        l[i] = li;
        if (l_h) l_h[i] = __float2half_rn(li);
        const float x = w * li;
#pragma unroll
        for (int k = 0; k < 3; ++k) g[k * N + i] = fmaf(x, ldf(gm + k * N + i), Av[k * N + i]);
    }
}

// b += w * l * gm (three components), the streaming form of the body force
// used when the state history is recomputed segment by segment
__global__ void k_bodyforce_acc(float *__restrict__ b, const float *__restrict__ l,
                                const float *__restrict__ gm, float w, long long N) {
    for (long long i = blockIdx.x * (long long)PT + threadIdx.x; i < N; i += (long long)gridDim.x * PT) {
        const float wl = w * l[i];
        b[i] = fmaf(wl, gm[i], b[i]);
        b[N + i] = fmaf(wl, gm[N + i], b[N + i]);
        b[2 * N + i] = fmaf(wl, gm[2 * N + i], b[2 * N + i]);
    }
}

// final condition of the adjoint for an upstream gradient:
// l = gmis * (m1 - m) - gm_final * inv_h3   (gm_final may be NULL)
__global__ void k_adjoint_final(float *__restrict__ l, const float *__restrict__ m1,
                                const float *__restrict__ m, const float *__restrict__ gmf,
                                float gmis, float inv_h3, long long N) {
    for (long long i = blockIdx.x * (long long)PT + threadIdx.x; i < N; i += (long long)gridDim.x * PT) {
        float r = gmis * (m1[i] - m[i]);
        if (gmf) r = fmaf(-inv_h3, gmf[i], r);
        l[i] = r;
    }
}


inline int grid1(long long N) {
    long long b = (N + PT - 1) / PT;
    return (int)(b < 152 * 16 ? b : 152 * 16);
}

}  // namespace

long long tile_count(const Dims &d) {
    return (long long)((d.n3 + PT3 - 1) / PT3) * ((d.n2 + PT2 - 1) / PT2) * ((d.n1 + PT1 - 1) / PT1);
}

void launch_tile_ranges(const Dims &d, const float *disp, int4 *tiles, cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_FOOTPOINT, st, 12.0 * d.N, 1);
    k_tile_ranges<<<pipe_blocks(d, 4), dim3(PT3, PT2), 0, st>>>(disp, d, tiles);
}

void launch_footpoints(const Dims &d, int nt, const float *v, float *dispm, float *dispp, int4 *tiles_m,
                       int4 *tiles_p, cudaStream_t st, Profiler *prof) {
    if (!dispm && !dispp) return;
    const float dt = 1.f / nt;
    const double two_pi = 6.283185307179586476925286766559;
    const float i1 = (float)(d.n1 / two_pi), i2 = (float)(d.n2 / two_pi), i3 = (float)(d.n3 / two_pi);
    if (d.iorder == 1) {
        {
            ProfScope ps(prof, CLAIRE_K_FOOTPOINT, st, (double)d.N * (12 + (dispm ? 12 : 0) + (dispp ? 12 : 0)), 1);
            const dim3 grid((d.n3 + BX - 1) / BX, (d.n2 + BY - 1) / BY, d.n1);
            k_footpoints<1><<<grid, dim3(BX, BY), 0, st>>>(v, dispm, dispp, d, dt, i1, i2, i3);
        }
        if (dispm) launch_tile_ranges(d, dispm, tiles_m, st, prof);
        if (dispp) launch_tile_ranges(d, dispp, tiles_p, st, prof);
        return;
    }
    ProfScope ps(prof, CLAIRE_K_FOOTPOINT, st, (double)d.N * (12 + (dispm ? 12 : 0) + (dispp ? 12 : 0)), 1);
    const size_t smem = 3 * BOX_FLOATS * sizeof(float);
    static SmemAttr attr;  // once per device
    attr.ensure(k_footpoints_box, (int)smem, "k_footpoints_box");
    k_footpoints_box<<<pipe_blocks(d, FP_OCC), dim3(PT3, PT2), smem, st>>>(v, dispm, dispp, d, dt, i1, i2, i3,
                                                                          chunk_ok(d, v), tiles_m, tiles_p);
}

void launch_interp(const Dims &d, const float *f, const float *disp, float *out, int4 *tiles,
                   cudaStream_t st, Profiler *prof, int kclass) {
    launch_tile_ranges(d, disp, tiles, st, prof);
    ProfScope ps(prof, kclass, st, 20.0 * d.N, kSlLaunches);
    SlArgs a{f, disp, out, nullptr, nullptr, nullptr, 0.f};
    launch_pipe<SL_PLAIN>(d, a, tiles, st);
}

void launch_adjoint_factor(const Dims &d, int nt, const float *divv, const float *dispp,
                           const int4 *tiles_p, float *cfac, cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_FOOTPOINT, st, 20.0 * d.N, kSlLaunches);
    SlArgs a{divv, dispp, cfac, divv, nullptr, nullptr, 1.f / nt};
    launch_pipe<SL_ADJFAC>(d, a, tiles_p, st);
}

void launch_state_step(const Dims &d, const float *src, const float *dispm, const int4 *tiles_m,
                       float *dst, cudaStream_t st, Profiler *prof, __half *dst_h) {
    ProfScope ps(prof, CLAIRE_K_STATE, st, (20.0 + (dst_h ? 2 : 0)) * d.N, kSlLaunches);
    SlArgs a{src, dispm, dst, nullptr, nullptr, nullptr, 0.f, dst_h};
    launch_pipe<SL_PLAIN>(d, a, tiles_m, st);
}

void launch_adjoint_step(const Dims &d, const float *src, const float *dispp, const int4 *tiles_p,
                         const float *cfac, float *dst, cudaStream_t st, Profiler *prof, int kclass,
                         __half *dst_h) {
    ProfScope ps(prof, kclass, st, (24.0 + (dst_h ? 2 : 0)) * d.N, kSlLaunches);
    SlArgs a{src, dispp, dst, cfac, nullptr, nullptr, 0.f, dst_h};
    launch_pipe<SL_ADJ>(d, a, tiles_p, st);
}

namespace {
template <typename TG>
void incstate_step(const Dims &d, float dt, const float *src, const float *dispm, const int4 *tiles_m,
                   const float *vt, const TG *gm_next, float *dst, cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_INCSTATE, st, (32.0 + 3 * sizeof(TG)) * d.N, kSlLaunches);
    SlArgsT<float, TG> a{src, dispm, dst, nullptr, vt, gm_next, dt};
    launch_pipe<SL_INCSTATE>(d, a, tiles_m, st);
}
template <typename TG>
void incstate_last(const Dims &d, float dt, const float *src, const float *dispm, const int4 *tiles_m,
                   const float *vt, const TG *gm_last, float *lt_last, float *mt_out, float *b_out,
                   cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_INCSTATE, st, (32.0 + 3 * sizeof(TG) + (mt_out ? 4 : 0) + (b_out ? 12 : 0)) * d.N,
                 kSlLaunches);
    SlArgsT<float, TG> a{src, dispm, lt_last, nullptr, vt, gm_last, dt};
    a.dst2 = mt_out;
    a.acc = b_out;
    launch_pipe<SL_INCLAST>(d, a, tiles_m, st);
}

template <typename TG>
void adjoint_acc(const Dims &d, const float *src, const float *dispp, const int4 *tiles_p, const float *cfac,
                 float *dst, const TG *gm, float *b, float w, bool want_dot, const float *p, double *partial,
                 const double *dot_add, double *dot_out, cudaStream_t st, Profiler *prof, int kclass,
                 __half *dst_h) {
    // p is read only by the step that forms the dot product
    ProfScope ps(prof, kclass, st, (48.0 + 3 * sizeof(TG) + (want_dot && p ? 12 : 0) + (dst_h ? 2 : 0)) * d.N,
                 kSlLaunches + (want_dot ? 1 : 0));
    SlArgsT<float, TG> a{src, dispp, dst, cfac, nullptr, gm, 0.f, dst_h};
    a.acc = b;
    a.w = w;
    if (want_dot) {
        a.pv = p;
        a.partial = partial;
        const int nb = launch_pipe<SL_ADJDOT>(d, a, tiles_p, st);
        launch_finalize(partial, nb, dot_add, dot_out, st);
    } else {
        launch_pipe<SL_ADJACC>(d, a, tiles_p, st);
    }
}
}  // namespace

void launch_incstate_last(const Dims &d, float dt, const float *src, const float *dispm, const int4 *tiles_m,
                          const float *vt, const float *gm_last, float *lt_last, float *mt_out, float *b_out,
                          cudaStream_t st, Profiler *prof) {
    incstate_last(d, dt, src, dispm, tiles_m, vt, gm_last, lt_last, mt_out, b_out, st, prof);
}
void launch_incstate_last(const Dims &d, float dt, const float *src, const float *dispm, const int4 *tiles_m,
                          const float *vt, const __half *gm_last, float *lt_last, float *mt_out, float *b_out,
                          cudaStream_t st, Profiler *prof) {
    incstate_last(d, dt, src, dispm, tiles_m, vt, gm_last, lt_last, mt_out, b_out, st, prof);
}

void launch_adjoint_acc(const Dims &d, const float *src, const float *dispp, const int4 *tiles_p, const float *cfac,
                        float *dst, const float *gm, float *b, float w, bool want_dot, const float *p,
                        double *partial, const double *dot_add, double *dot_out, cudaStream_t st, Profiler *prof,
                        int kclass, __half *dst_h) {
    adjoint_acc(d, src, dispp, tiles_p, cfac, dst, gm, b, w, want_dot, p, partial, dot_add, dot_out, st, prof,
                kclass, dst_h);
}
void launch_adjoint_acc(const Dims &d, const float *src, const float *dispp, const int4 *tiles_p, const float *cfac,
                        float *dst, const __half *gm, float *b, float w, bool want_dot, const float *p,
                        double *partial, const double *dot_add, double *dot_out, cudaStream_t st, Profiler *prof,
                        int kclass, __half *dst_h) {
    adjoint_acc(d, src, dispp, tiles_p, cfac, dst, gm, b, w, want_dot, p, partial, dot_add, dot_out, st, prof,
                kclass, dst_h);
}

void launch_incstate_init(const Dims &d, float dt, const float *vt, const float *gm0, float *u0,
                          cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_VECTOR, st, 28.0 * d.N);
    k_incstate_init<<<grid1(d.N), PT, 0, st>>>(vt, gm0, u0, d.N, 0.5f * dt);
}
void launch_incstate_init(const Dims &d, float dt, const float *vt, const __half *gm0, float *u0,
                          cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_VECTOR, st, 22.0 * d.N);
    k_incstate_init<<<grid1(d.N), PT, 0, st>>>(vt, gm0, u0, d.N, 0.5f * dt);
}

void launch_incstate_step(const Dims &d, float dt, const float *src, const float *dispm,
                          const int4 *tiles_m, const float *vt, const float *gm_next, float *dst,
                          cudaStream_t st, Profiler *prof) {
    incstate_step(d, dt, src, dispm, tiles_m, vt, gm_next, dst, st, prof);
}
void launch_incstate_step(const Dims &d, float dt, const float *src, const float *dispm,
                          const int4 *tiles_m, const float *vt, const __half *gm_next, float *dst,
                          cudaStream_t st, Profiler *prof) {
    incstate_step(d, dt, src, dispm, tiles_m, vt, gm_next, dst, st, prof);
}

namespace {
template <typename TG>
void adjfinal_acc(const Dims &d, const float *m1, const float *m, float *l, __half *l_h, const TG *gm,
                  const float *Av, float *g, float w, cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_BODYFORCE, st, (36.0 + 3 * sizeof(TG) + (l_h ? 2 : 0)) * d.N);
    k_adjfinal_acc<<<grid1(d.N), PT, 0, st>>>(m1, m, l, l_h, gm, Av, g, w, d.N);
}
}  // namespace

void launch_adjfinal_acc(const Dims &d, const float *m1, const float *m, float *l, __half *l_h, const float *gm,
                         const float *Av, float *g, float w, cudaStream_t st, Profiler *prof) {
    adjfinal_acc(d, m1, m, l, l_h, gm, Av, g, w, st, prof);
}
void launch_adjfinal_acc(const Dims &d, const float *m1, const float *m, float *l, __half *l_h, const __half *gm,
                         const float *Av, float *g, float w, cudaStream_t st, Profiler *prof) {
    adjfinal_acc(d, m1, m, l, l_h, gm, Av, g, w, st, prof);
}

void launch_bodyforce_acc(const Dims &d, float *b, const float *l, const float *gm, float w,
                          cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_BODYFORCE, st, 40.0 * d.N);
    k_bodyforce_acc<<<grid1(d.N), PT, 0, st>>>(b, l, gm, w, d.N);
}

void launch_adjoint_final(const Dims &d, float *l, const float *m1, const float *m,
                          const float *gm_final, float gmis, float inv_h3, cudaStream_t st,
                          Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_VECTOR, st, (double)d.N * (gm_final ? 16 : 12));
    k_adjoint_final<<<grid1(d.N), PT, 0, st>>>(l, m1, m, gm_final, gmis, inv_h3, d.N);
}

}  // namespace claire

// Violations counted by the debug build's box checks since the last reset
// (CLAIRE_ERR_STATE in the release build, which has no counter).
extern "C" int claire_check_count(unsigned long long *count, int reset) {
    if (!count) return CLAIRE_ERR_ARG;
#ifdef CLAIRE_CHECKS
    if (cudaDeviceSynchronize() != cudaSuccess) return CLAIRE_ERR_CUDA;
    if (cudaMemcpyFromSymbol(count, claire::g_check_count, sizeof(*count)) != cudaSuccess) return CLAIRE_ERR_CUDA;
    if (reset) {
        const unsigned long long z = 0;
        if (cudaMemcpyToSymbol(claire::g_check_count, &z, sizeof(z)) != cudaSuccess) return CLAIRE_ERR_CUDA;
    }
    return CLAIRE_OK;
#else
    (void)reset;
    *count = 0;
    return CLAIRE_ERR_STATE;
#endif
}
