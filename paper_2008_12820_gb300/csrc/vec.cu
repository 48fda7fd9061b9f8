// vec.cu -- FP64-accumulated reductions and fused vector updates for PCG and
// the Gauss-Newton step (paper Algorithm 1; Eq. 3.3).
//
// Reductions: FP64 is slow on this part, so a thread does not widen every
// element.  It accumulates its grid-stride range with error-free
// transformations in FP32 (Acc2, reduce.cuh), as accurate as summing in twice
// the working precision; the pair (sum, compensation) is widened to FP64
// once, a block reduces in FP64 by warp shuffles, block partials go to a
// fixed-size array, and one block sums them in a fixed order: deterministic
// for a given grid.
#include <cuda_fp16.h>
#include <cstdint>
#include <cuda_runtime.h>

#include "claire_internal.cuh"
#include "reduce.cuh"

namespace claire {

namespace {

__device__ __forceinline__ float ldv(const float *p) { return *p; }
__device__ __forceinline__ float ldv(const __half *p) { return __half2float(*p); }

constexpr int RT = 256;

// block sum of v (1D blocks of RT threads); valid in thread 0
__device__ __forceinline__ double block_sum(double v) { return block_sum_n<RT>(v, threadIdx.x); }

// Four consecutive elements at once (16-byte loads and stores) where the
// length is a multiple of 4 and the pointers are 16-byte aligned: four times
// the bytes in flight per instruction, which the scalar grid-stride loops
// lack to cover HBM latency.  Element k of a float4 as an lvalue (k is a
// compile-time constant after unrolling).
__device__ __forceinline__ float &lane(float4 &v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w)); }
__device__ __forceinline__ float4 ld4(const float *p, long long i) { return reinterpret_cast<const float4 *>(p)[i]; }
__device__ __forceinline__ float4 ld4(const __half *p, long long i) {
    const uint2 u = reinterpret_cast<const uint2 *>(p)[i];
    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void st4(float *p, long long i, const float4 &v) { reinterpret_cast<float4 *>(p)[i] = v; }

// MODE 0: sum a*b;  MODE 1: sum (a-b)^2
template <int MODE>
__device__ __forceinline__ void reduce2_add(Acc2 &acc, float x, float y) {
    if (MODE == 0) {
        acc.add_prod(x, y);
    } else {
        // d = x - y exactly as dh + dl (TwoSum), then d^2 ~ dh^2 + 2 dh dl
        const float dh = __fsub_rn(x, y);
        const float z = __fsub_rn(dh, x);
        const float dl = __fadd_rn(__fsub_rn(x, __fsub_rn(dh, z)), __fsub_rn(-y, z));
        const float p = __fmul_rn(dh, dh);
        acc.add(p, fmaf(dh, dh, -p) + 2.f * dh * dl);
    }
}

template <int MODE, typename TA = float, bool V4 = false>
__global__ void __launch_bounds__(RT) k_reduce2(const TA *__restrict__ a, const float *__restrict__ b,
                                                long long n, double *__restrict__ partial) {
    Acc2 acc;
    const long long stride = (long long)gridDim.x * RT;
    if (V4) {
        for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < (n >> 2); i += stride) {
            float4 x = ld4(a, i), y = ld4(b, i);
#pragma unroll
            for (int k = 0; k < 4; ++k) reduce2_add<MODE>(acc, lane(x, k), lane(y, k));
        }
    } else {
        for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += stride)
            reduce2_add<MODE>(acc, ldv(a + i), b[i]);
    }
    double s = block_sum(acc.value());
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(RT) k_finalize(const double *__restrict__ partial, int nb,
                                                 double *__restrict__ out, const double *__restrict__ add = nullptr) {
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += RT) s += partial[i];
    s = block_sum(s);
    if (threadIdx.x == 0) out[0] = add ? s + add[0] : s;
}

// x += alpha p ; r -= alpha q ; partial sums of r.r
__global__ void __launch_bounds__(RT) k_pcg_xr(float *__restrict__ x, float *__restrict__ r,
                                               const float *__restrict__ p, const float *__restrict__ q,
                                               float alpha, long long n, double *__restrict__ partial) {
    Acc2 acc;
    const long long stride = (long long)gridDim.x * RT;
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += stride) {
        x[i] = fmaf(alpha, p[i], x[i]);
        const float ri = fmaf(-alpha, q[i], r[i]);
        r[i] = ri;
        acc.add_prod(ri, ri);
    }
    double s = block_sum(acc.value());
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(RT) k_pcg_p(float *__restrict__ p, const float *__restrict__ z,
                                              float beta, long long n) {
    const long long stride = (long long)gridDim.x * RT;
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += stride)
        p[i] = fmaf(beta, p[i], z[i]);
}

__global__ void __launch_bounds__(RT) k_axpby(float *__restrict__ out, float a, const float *__restrict__ x,
                                              float b, const float *__restrict__ y, long long n) {
    const long long stride = (long long)gridDim.x * RT;
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += stride)
        out[i] = y ? fmaf(a, x[i], b * y[i]) : a * x[i];
}

__global__ void __launch_bounds__(RT) k_diff_flag(const float *__restrict__ a, const float *__restrict__ b,
                                                  long long n, int *__restrict__ flag) {
    const long long stride = (long long)gridDim.x * RT;
    bool diff = false;
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += stride)
        diff |= (__float_as_uint(a[i]) != __float_as_uint(b[i]));
    if (__syncthreads_or(diff) && threadIdx.x == 0) atomicOr(flag, 1);
}

// four block sums at once (one barrier round)
__device__ __forceinline__ void block_sum4(double v[4]) {
    __shared__ double ws4[4][RT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = warp_sum(v[k]);
        if (lane == 0) ws4[k][w] = v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double t = (w == 0 && lane < RT / 32) ? ws4[k][lane] : 0.0;
        v[k] = w == 0 ? warp_sum(t) : 0.0;
    }
}

// statistics of a vector field r [3][N]: r.r and the sum of each component
__device__ __forceinline__ void stats_store(Acc2 &rr, Acc2 *sc, double *partial) {
    double v[4] = {rr.value(), sc[0].value(), sc[1].value(), sc[2].value()};
    block_sum4(v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) partial[4 * blockIdx.x + k] = v[k];
    }
}

template <bool V4>
__global__ void __launch_bounds__(RT) k_stats(const float *__restrict__ r, long long N,
                                              double *__restrict__ partial) {
    Acc2 rr, sc[3];
    const long long stride = (long long)gridDim.x * RT;
    if (V4) {
        const long long N4 = N >> 2;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < N4; i += stride) {
                float4 rv = ld4(r, c * N4 + i);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    rr.add_prod(lane(rv, k), lane(rv, k));
                    sc[c].add(lane(rv, k), 0.f);
                }
            }
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c)
            for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < N; i += stride) {
                const float ri = r[c * N + i];
                rr.add_prod(ri, ri);
                sc[c].add(ri, 0.f);
            }
    }
    stats_store(rr, sc, partial);
}

// PCG update with the regularization term carried along (x, A x, r):
// x += a p; Ax += a Ap; r -= a q; statistics of the new r.  q_adds_Ap: q
// holds only the body force of H p, and H p = Ap + q is formed here.
// dpq, drz (optional): the step length is alpha = rz / pq from device
// memory (no host round trip); with pq <= 0 or non-finite nothing is updated
// (negative curvature: the caller stops) and the statistics are those of the
// unchanged r.  pq_out keeps pq for the caller.
template <bool V4>
__global__ void __launch_bounds__(RT) k_pcg_update(float *__restrict__ x, float *__restrict__ Ax,
                                                   float *__restrict__ r, const float *__restrict__ p,
                                                   const float *__restrict__ Ap,
                                                   const float *__restrict__ q, float alpha,
                                                   long long N, double *__restrict__ partial, int q_adds_Ap,
                                                   const double *__restrict__ dpq, const double *__restrict__ drz,
                                                   double *__restrict__ pq_out) {
    Acc2 rr, sc[3];
    const long long stride = (long long)gridDim.x * RT;
    const bool wantAp = Ax || q_adds_Ap;
    bool upd = true;
    if (dpq) {
        const double pq = *dpq;
        upd = pq > 0.0 && pq <= 1.7976931348623157e308;
        alpha = upd ? (float)(*drz / pq) : 0.f;
        if (pq_out && blockIdx.x == 0 && threadIdx.x == 0) *pq_out = pq;
    }
    if (V4) {
        const long long N4 = N >> 2;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            for (long long i = c * N4 + blockIdx.x * (long long)RT + threadIdx.x; i < (c + 1) * N4; i += stride) {
                float4 xv = ld4(x, i), rv = ld4(r, i);
                const float4 pv = ld4(p, i), qv = ld4(q, i);
                const float4 apv = wantAp ? ld4(Ap, i) : make_float4(0.f, 0.f, 0.f, 0.f);
                float4 axv = Ax ? ld4(Ax, i) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    float4 pk = pv, qk = qv, ak = apv;
                    lane(xv, k) = fmaf(alpha, lane(pk, k), lane(xv, k));
                    lane(axv, k) = fmaf(alpha, lane(ak, k), lane(axv, k));
                    const float qi = q_adds_Ap ? lane(qk, k) + lane(ak, k) : lane(qk, k);
                    const float ri = upd ? fmaf(-alpha, qi, lane(rv, k)) : lane(rv, k);
                    lane(rv, k) = ri;
                    rr.add_prod(ri, ri);
                    sc[c].add(ri, 0.f);
                }
                if (upd) {
                    st4(x, i, xv);
                    if (Ax) st4(Ax, i, axv);
                    st4(r, i, rv);
                }
            }
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c)
            for (long long i = c * N + blockIdx.x * (long long)RT + threadIdx.x; i < (c + 1) * N; i += stride) {
                float ri = r[i];
                if (upd) {
                    x[i] = fmaf(alpha, p[i], x[i]);
                    const float Api = wantAp ? Ap[i] : 0.f;
                    if (Ax) Ax[i] = fmaf(alpha, Api, Ax[i]);
                    const float qi = q_adds_Ap ? q[i] + Api : q[i];
                    ri = fmaf(-alpha, qi, ri);
                    r[i] = ri;
                }
                rr.add_prod(ri, ri);
                sc[c].add(ri, 0.f);
            }
    }
    stats_store(rr, sc, partial);
}

// the four line-search dot products in one sweep over g, x, Av, v, Ax
__global__ void __launch_bounds__(RT) k_ls_dots(const float *__restrict__ g, const float *__restrict__ x,
                                                const float *__restrict__ Av, const float *__restrict__ v,
                                                const float *__restrict__ Ax, long long n,
                                                double *__restrict__ partial) {
    Acc2 a0, a1, a2, a3;
    const long long stride = (long long)gridDim.x * RT;
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += stride) {
        const float xi = x[i], Axi = Ax[i];
        a0.add_prod(g[i], xi);
        a1.add_prod(xi, Av[i]);
        a2.add_prod(v[i], Axi);
        a3.add_prod(xi, Axi);
    }
    double s[4] = {a0.value(), a1.value(), a2.value(), a3.value()};
    block_sum4(s);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) partial[4 * blockIdx.x + k] = s[k];
}

__global__ void __launch_bounds__(RT) k_finalize4(const double *__restrict__ partial, int nb,
                                                  double *__restrict__ out) {
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < nb; i += RT)
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] += partial[4 * i + k];
    block_sum4(v);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) out[k] = v[k];
}

// new search direction and its image under beta*A without an FFT:
//   p = z + b p,   Ap = (r - mean r) + b Ap
// since beta*A z = r - mean(r) for z = (beta*A)^{-1} r (the inverse is the
// identity on the zero wavenumber, where beta*A vanishes).  init: b = 0 and
// the old p, Ap are not read.  rsum: device sums of the components of r.
// With a preconditioner other than (beta*A)^{-1}, Az (= beta*A z, applied
// spectrally by the caller) replaces r - mean r.
__global__ void __launch_bounds__(RT) k_pcg_dir(float *__restrict__ p, float *__restrict__ Ap,
                                                const float *__restrict__ z, const float *__restrict__ r,
                                                const double *__restrict__ rsum, const float *__restrict__ Az,
                                                float b, long long N, int init, const double *__restrict__ dbn,
                                                const double *__restrict__ dbd) {
    const long long stride = (long long)gridDim.x * RT;
    // dbn, dbd (optional): b = num / den from device memory
    if (dbn) b = (float)(*dbn / *dbd);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float mean = Az ? 0.f : (float)(rsum[c] / (double)N);
        for (long long i = c * N + blockIdx.x * (long long)RT + threadIdx.x; i < (c + 1) * N; i += stride) {
            const float ar = Az ? Az[i] : r[i] - mean;
            if (init) {
                p[i] = z[i];
                Ap[i] = ar;
            } else {
                p[i] = fmaf(b, p[i], z[i]);
                Ap[i] = fmaf(b, Ap[i], ar);
            }
        }
    }
}

// k_pcg_dir per voxel, also writing the first incremental-state field of the
// next matvec, u0 = dt/2 f^0 with f^0 = -p . grad m^0 (saves that pass)
// four blocks per SM (64 registers, no spills): 6.66 -> 6.31 ms of PCG vector
// updates per 256^3 solve against three blocks at 80 registers
template <typename TG, bool V4>
__global__ void __launch_bounds__(RT, 4) k_pcg_dir_u0(float *__restrict__ p, float *__restrict__ Ap,
                                                   const float *__restrict__ z, const float *__restrict__ r,
                                                   const double *__restrict__ rsum, const float *__restrict__ Az,
                                                   float b, long long N, int init, const TG *__restrict__ gm0,
                                                   float *__restrict__ u0, float hdt,
                                                   double *__restrict__ partial, const double *__restrict__ dbn,
                                                   const double *__restrict__ dbd) {
    const long long stride = (long long)gridDim.x * RT;
    // dbn, dbd (optional): b = num / den from device memory (the PCG ratio of
    // successive r . z, without a host round trip)
    if (dbn) b = (float)(*dbn / *dbd);
    Acc2 pap;
    float mean[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) mean[c] = Az ? 0.f : (float)(rsum[c] / (double)N);
    if (V4) {
        const long long N4 = N >> 2;
        for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < N4; i += stride) {
            float4 pc[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const long long k4 = c * N4 + i;
                float4 arv = Az ? ld4(Az, k4) : ld4(r, k4);
                const float4 zv = ld4(z, k4);
                float4 pv = init ? zv : ld4(p, k4);
                float4 apv = init ? arv : ld4(Ap, k4);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    float4 zk = zv;
                    const float ar = Az ? lane(arv, k) : lane(arv, k) - mean[c];
                    float apc;
                    if (init) {
                        apc = ar;
                    } else {
                        lane(pv, k) = fmaf(b, lane(pv, k), lane(zk, k));
                        apc = fmaf(b, lane(apv, k), ar);
                    }
                    lane(apv, k) = apc;
                    if (partial) pap.add_prod(lane(pv, k), apc);
                }
                st4(Ap, k4, apv);
                st4(p, k4, pv);
                pc[c] = pv;
            }
            const float4 g0 = ld4(gm0, i), g1 = ld4(gm0 + N, i), g2 = ld4(gm0 + 2 * N, i);
            float4 uv;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float4 a0 = g0, a1 = g1, a2 = g2;
                const float f = -(lane(pc[0], k) * lane(a0, k) + lane(pc[1], k) * lane(a1, k) +
                                  lane(pc[2], k) * lane(a2, k));
                lane(uv, k) = hdt * f;
            }
            st4(u0, i, uv);
        }
    } else {
        for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < N; i += stride) {
            float pc[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const long long k = c * N + i;
                const float ar = Az ? Az[k] : r[k] - mean[c];
                float apc;
                if (init) {
                    pc[c] = z[k];
                    apc = ar;
                } else {
                    pc[c] = fmaf(b, p[k], z[k]);
                    apc = fmaf(b, Ap[k], ar);
                }
                Ap[k] = apc;
                p[k] = pc[c];
                if (partial) pap.add_prod(pc[c], apc);
            }
            const float f = -(pc[0] * ldv(gm0 + i) + pc[1] * ldv(gm0 + N + i) + pc[2] * ldv(gm0 + 2 * N + i));
            u0[i] = hdt * f;
        }
    }
    if (partial) {
        const double s = block_sum(pap.value());
        if (threadIdx.x == 0) partial[blockIdx.x] = s;
    }
}

// zero-velocity Hessian applied to p given beta0*A p:  q = Ap + gm (gm . p)
__global__ void __launch_bounds__(RT) k_h0_apply(float *__restrict__ q, const float *__restrict__ Ap,
                                                 const float *__restrict__ gm, const float *__restrict__ p,
                                                 long long N) {
    const long long stride = (long long)gridDim.x * RT;
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < N; i += stride) {
        const float g1 = gm[i], g2 = gm[N + i], g3 = gm[2 * N + i];
        const float gp = g1 * p[i] + g2 * p[N + i] + g3 * p[2 * N + i];
        q[i] = fmaf(g1, gp, Ap[i]);
        q[N + i] = fmaf(g2, gp, Ap[N + i]);
        q[2 * N + i] = fmaf(g3, gp, Ap[2 * N + i]);
    }
}

// Body force of the Hessian matvec plus the carried beta*A p, and p . q:
//   q_d = Ap_d + dt sum_j w_j l^j d_d m^j,   partial sums of sum_d p_d q_d
// (fuses the PCG curvature product into the pass that writes q)
__global__ void k_f2h(const float *__restrict__ in, __half *__restrict__ out, long long n) {
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT)
        out[i] = __float2half_rn(in[i]);
}
__global__ void k_h2f(const __half *__restrict__ in, float *__restrict__ out, long long n) {
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT)
        out[i] = __half2float(in[i]);
}

inline int blocks_for(long long n) {
    long long b = (n + RT - 1) / RT;
    return (int)(b < kReduceBlocks ? b : kReduceBlocks);
}

// the float4 forms apply: a whole number of float4 per component and every
// pointer 16-byte aligned (8-byte for FP16 fields); null pointers pass
template <typename T>
inline bool al16(const T *p) { return ((uintptr_t)p & (sizeof(T) == 2 ? 7 : 15)) == 0; }
inline bool v4_ok(long long N) { return (N & 3) == 0; }
template <typename T, typename... R>
inline bool v4_ok(long long N, const T *p, const R *...rest) { return al16(p) && v4_ok(N, rest...); }

}  // namespace

void launch_finalize(const double *partial, int nb, const double *add, double *dev_out, cudaStream_t st) {
    k_finalize<<<1, RT, 0, st>>>(partial, nb, dev_out, add);
}

void launch_ls_dots(const float *g, const float *x, const float *Av, const float *v, const float *Ax, long long n,
                    double *partial, double *dev_out, cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_REDUCE, st, 20.0 * n, 2);
    const int nb = blocks_for(n);
    k_ls_dots<<<nb, RT, 0, st>>>(g, x, Av, v, Ax, n, partial);
    k_finalize4<<<1, RT, 0, st>>>(partial, nb, dev_out);
}

void launch_dot(const float *a, const float *b, long long n, double *partial, double *dev_out,
                cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_REDUCE, st, 8.0 * n, 2);
    const bool v4 = v4_ok(n, a, b);
    const int nb = blocks_for(v4 ? n / 4 : n);
    if (v4) k_reduce2<0, float, true><<<nb, RT, 0, st>>>(a, b, n, partial);
    else k_reduce2<0><<<nb, RT, 0, st>>>(a, b, n, partial);
    k_finalize<<<1, RT, 0, st>>>(partial, nb, dev_out);
}

void launch_sqdiff(const float *a, const float *b, long long n, double *partial, double *dev_out,
                   cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_REDUCE, st, 8.0 * n, 2);
    const bool v4 = v4_ok(n, a, b);
    const int nb = blocks_for(v4 ? n / 4 : n);
    if (v4) k_reduce2<1, float, true><<<nb, RT, 0, st>>>(a, b, n, partial);
    else k_reduce2<1><<<nb, RT, 0, st>>>(a, b, n, partial);
    k_finalize<<<1, RT, 0, st>>>(partial, nb, dev_out);
}

void launch_f2h(const float *in, __half *out, long long n, cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_VECTOR, st, 6.0 * n);
    k_f2h<<<blocks_for(n), RT, 0, st>>>(in, out, n);
}

void launch_h2f(const __half *in, float *out, long long n, cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_VECTOR, st, 6.0 * n);
    k_h2f<<<blocks_for(n), RT, 0, st>>>(in, out, n);
}

void launch_pcg_xr(float *x, float *r, const float *p, const float *q, float alpha, long long n,
                   double *partial, double *dev_out, cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_VECTOR, st, 24.0 * n, 2);
    const int nb = blocks_for(n);
    k_pcg_xr<<<nb, RT, 0, st>>>(x, r, p, q, alpha, n, partial);
    k_finalize<<<1, RT, 0, st>>>(partial, nb, dev_out);
}

void launch_pcg_p(float *p, const float *z, float beta, long long n, cudaStream_t st,
                  Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_VECTOR, st, 12.0 * n);
    k_pcg_p<<<blocks_for(n), RT, 0, st>>>(p, z, beta, n);
}

void launch_axpby(float *out, float a, const float *x, float b, const float *y, long long n,
                  cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_VECTOR, st, (y ? 12.0 : 8.0) * n);
    k_axpby<<<blocks_for(n), RT, 0, st>>>(out, a, x, b, y, n);
}

void launch_diff_flag(const float *a, const float *b, long long n, int *flag, cudaStream_t st,
                      Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_VECTOR, st, 8.0 * n);
    cudaMemsetAsync(flag, 0, sizeof(int), st);
    k_diff_flag<<<blocks_for(n), RT, 0, st>>>(a, b, n, flag);
}

void launch_stats(const float *r, long long N, double *partial, double *dev_out, cudaStream_t st,
                  Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_REDUCE, st, 12.0 * N, 2);
    const bool v4 = v4_ok(N, r);
    const int nb = blocks_for(v4 ? N / 4 : N);
    if (v4) k_stats<true><<<nb, RT, 0, st>>>(r, N, partial);
    else k_stats<false><<<nb, RT, 0, st>>>(r, N, partial);
    k_finalize4<<<1, RT, 0, st>>>(partial, nb, dev_out);
}

void launch_pcg_update(float *x, float *Ax, float *r, const float *p, const float *Ap,
                       const float *q, float alpha, long long N, double *partial, double *dev_out,
                       cudaStream_t st, Profiler *prof, bool q_adds_Ap, const double *dpq, const double *drz,
                       double *pq_out) {
    ProfScope ps(prof, CLAIRE_K_VECTOR, st, 3.0 * N * (Ax ? 36 : 24), 2);
    const bool v4 = v4_ok(N, x, Ax, r, p, Ap, q);
    const int nb = blocks_for(v4 ? N / 4 : N);
    if (v4)
        k_pcg_update<true><<<nb, RT, 0, st>>>(x, Ax, r, p, Ap, q, alpha, N, partial, q_adds_Ap ? 1 : 0, dpq, drz,
                                             pq_out);
    else
        k_pcg_update<false><<<nb, RT, 0, st>>>(x, Ax, r, p, Ap, q, alpha, N, partial, q_adds_Ap ? 1 : 0, dpq, drz,
                                              pq_out);
    k_finalize4<<<1, RT, 0, st>>>(partial, nb, dev_out);
}

void launch_pcg_dir(float *p, float *Ap, const float *z, const float *r, const double *rsum,
                    const float *Az, float b, long long N, bool init, cudaStream_t st,
                    Profiler *prof, const double *dbn, const double *dbd) {
    ProfScope ps(prof, CLAIRE_K_VECTOR, st, 3.0 * N * (init ? 16 : 24));
    k_pcg_dir<<<blocks_for(3 * N), RT, 0, st>>>(p, Ap, z, r, rsum, Az, b, N, init ? 1 : 0, dbn, dbd);
}

// ---- device-side control of the inner PCG of the H0 preconditioners -----
// c: the inner solve's device scalars (see launch_inner_*): c[0] tolerance,
// c[1] ||r0||, c[2] p.q, c[3] r.z of the current direction, c[4] r.z of the
// new residual, c[5] iterations, c[6..9] ||r||^2 and the component sums of r,
// c[10] loop bodies run.
namespace {
__global__ void k_inner_init(double *c) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        c[1] = sqrt(c[6]);
        c[5] = 0.0;
        c[10] = 0.0;
    }
}
// after the PCG update of one loop body: the same decisions, in the same
// FP64 arithmetic, as the host-driven loop (stop on p.q <= 0 without counting
// the step; otherwise count it and stop when ||r|| <= tol ||r0|| -- unless
// the iteration count is fixed -- or at maxit), and the while condition
__global__ void k_inner_ctl(double *c, cudaGraphConditionalHandle h, cudaGraphConditionalHandle h_tail, int maxit,
                            int fixed) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        c[10] += 1.0;
        unsigned int cont = 0;
        const double pq = c[2];
        if (pq > 0.0) {
            const double it = c[5] + 1.0;
            c[5] = it;
            const double rn = sqrt(c[6]);
            const bool conv = !fixed && rn <= c[0] * c[1];
            cont = (!conv && it < (double)maxit) ? 1u : 0u;
        }
        cudaGraphSetConditional(h, cont);
        cudaGraphSetConditional(h_tail, cont);
    }
}
// after the PCG update of one outer loop body: the decisions of the
// host-driven loop in the same FP64 arithmetic.  d: the solver's result
// slots (d[0] ||r||^2 after the update, d[12] p.Hp); c: the loop's scalars
// (c[0] stopping threshold eps_K ||r0||, c[1] iterations, c[2] flags: 1
// non-finite p.Hp, 2 non-positive curvature in the first iteration, c[3]
// bodies run).  Non-finite p.Hp stops the loop; p.Hp <= 0 counts the step and
// stops (the update changed nothing); otherwise count and test.
__global__ void k_pcg_ctl(const double *d, double *c, cudaGraphConditionalHandle h, cudaGraphConditionalHandle h_tail,
                          int maxit, int fixed) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        c[3] += 1.0;
        const double pq = d[12];
        unsigned int cont = 0;
        if (!(pq >= -1.7976931348623157e308 && pq <= 1.7976931348623157e308)) {
            c[2] = 1.0;
        } else if (!(pq > 0.0)) {
            if (c[1] == 0.0) c[2] = 2.0;
            c[1] += 1.0;
        } else {
            const double it = c[1] + 1.0;
            c[1] = it;
            const double rn = sqrt(d[0]);
            const bool conv = !fixed && rn <= c[0];
            cont = (!conv && it < (double)maxit) ? 1u : 0u;
        }
        cudaGraphSetConditional(h, cont);
        cudaGraphSetConditional(h_tail, cont);
    }
}
// negative curvature in the first PCG iteration keeps the preconditioned
// residual: x = z, Ax = Ap (flag c[2] == 2, set by k_pcg_ctl); otherwise a
// no-op
__global__ void k_pcg_negcopy(const double *c, float *__restrict__ x, float *__restrict__ Ax,
                              const float *__restrict__ z, const float *__restrict__ Ap, long long n) {
    if (c[2] != 2.0) return;
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT) {
        x[i] = z[i];
        Ax[i] = Ap[i];
    }
}
__global__ void k_pcg_ctl_init(double *c, double thr) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        c[0] = thr;
        c[1] = c[2] = c[3] = 0.0;
    }
}

__global__ void k_scalar_copy(double *dst, const double *src) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *dst = *src;
}
__global__ void k_scalar_set(double *dst, double v) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *dst = v;
}
}  // namespace

void launch_inner_init(double *c, cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_REDUCE, st);
    k_inner_init<<<1, 32, 0, st>>>(c);
}
void launch_inner_ctl(double *c, cudaGraphConditionalHandle h, cudaGraphConditionalHandle h_tail, int maxit,
                      bool fixed, cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_REDUCE, st);
    k_inner_ctl<<<1, 32, 0, st>>>(c, h, h_tail, maxit, fixed ? 1 : 0);
}
void launch_pcg_ctl(const double *d, double *c, cudaGraphConditionalHandle h, cudaGraphConditionalHandle h_tail,
                    int maxit, bool fixed, cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_REDUCE, st);
    k_pcg_ctl<<<1, 32, 0, st>>>(d, c, h, h_tail, maxit, fixed ? 1 : 0);
}
void launch_pcg_negcopy(const double *c, float *x, float *Ax, const float *z, const float *Ap, long long n,
                        cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_VECTOR, st);
    k_pcg_negcopy<<<blocks_for(n), RT, 0, st>>>(c, x, Ax, z, Ap, n);
}
void launch_pcg_ctl_init(double *c, double thr, cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_REDUCE, st);
    k_pcg_ctl_init<<<1, 32, 0, st>>>(c, thr);
}
void launch_scalar_copy(double *dst, const double *src, cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_REDUCE, st);
    k_scalar_copy<<<1, 32, 0, st>>>(dst, src);
}
void launch_scalar_set(double *dst, double v, cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_REDUCE, st);
    k_scalar_set<<<1, 32, 0, st>>>(dst, v);
}

template <typename TG>
static void pcg_dir_u0(float *p, float *Ap, const float *z, const float *r, const double *rsum, const float *Az,
                       float b, long long N, bool init, const TG *gm0, float *u0, float hdt, double *partial,
                       double *pap_out, cudaStream_t st, Profiler *prof, const double *dbn, const double *dbd) {
    ProfScope ps(prof, CLAIRE_K_VECTOR, st, (double)N * (3.0 * (init ? 16 : 24) + 3 * sizeof(TG) + 4),
                 pap_out ? 2 : 1);
    const bool v4 = v4_ok(N, p, Ap, z, r, Az, gm0, u0);
    const int nb = blocks_for(v4 ? N / 4 : N);
    if (v4)
        k_pcg_dir_u0<TG, true><<<nb, RT, 0, st>>>(p, Ap, z, r, rsum, Az, b, N, init ? 1 : 0, gm0, u0, hdt,
                                                  pap_out ? partial : nullptr, dbn, dbd);
    else
        k_pcg_dir_u0<TG, false><<<nb, RT, 0, st>>>(p, Ap, z, r, rsum, Az, b, N, init ? 1 : 0, gm0, u0, hdt,
                                                   pap_out ? partial : nullptr, dbn, dbd);
    if (pap_out) k_finalize<<<1, RT, 0, st>>>(partial, nb, pap_out);
}

void launch_pcg_dir_u0(float *p, float *Ap, const float *z, const float *r, const double *rsum, const float *Az,
                       float b, long long N, bool init, const float *gm0, float *u0, float hdt, double *partial,
                       double *pap_out, cudaStream_t st, Profiler *prof, const double *dbn, const double *dbd) {
    pcg_dir_u0(p, Ap, z, r, rsum, Az, b, N, init, gm0, u0, hdt, partial, pap_out, st, prof, dbn, dbd);
}
void launch_pcg_dir_u0(float *p, float *Ap, const float *z, const float *r, const double *rsum, const float *Az,
                       float b, long long N, bool init, const __half *gm0, float *u0, float hdt, double *partial,
                       double *pap_out, cudaStream_t st, Profiler *prof, const double *dbn, const double *dbd) {
    pcg_dir_u0(p, Ap, z, r, rsum, Az, b, N, init, gm0, u0, hdt, partial, pap_out, st, prof, dbn, dbd);
}

void launch_h0_apply(float *q, const float *Ap, const float *gm, const float *p, long long N,
                     cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_VECTOR, st, 48.0 * N);
    k_h0_apply<<<blocks_for(N), RT, 0, st>>>(q, Ap, gm, p, N);
}

}  // namespace claire
