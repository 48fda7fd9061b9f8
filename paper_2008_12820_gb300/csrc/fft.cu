// fft.cu -- shared-memory pencil 3D FFT with fused spectral multipliers
// (paper Section 3, "Discretization": the vector Laplacian, the divergence
// penalty and their inverse are diagonal in Fourier space; first derivatives
// are spectral as well).
//
// A spectral operator out = F^-1[ M(k) F in ] runs as five pencil passes, each
// reading and writing HBM once:
//   1. x3 forward, real -> half spectrum.  Two real lines are packed into one
//      complex line, transformed, and separated by Hermitian symmetry.
//   2. x2 forward, complex, in place.
//   3. x1 forward, multiplier M(k) for all components at once (the divergence
//      penalty couples them), x1 inverse; in place.
//   4. x2 inverse, in place.
//   5. x3 inverse, half spectrum -> real, two lines per complex transform,
//      with an optional addend in the epilogue.
// Each pass stages a tile of whole lines in shared memory and runs a
// mixed-radix (2, 3, 4, 5) Stockham FFT there: natural-order output, no bit
// reversal, twiddles from a table computed in double on the host.
// Strided passes (x2, x1) load tiles of TK consecutive k3 columns so that
// every row access is a contiguous 8*TK-byte segment.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "claire_internal.cuh"
#include "fft_core.cuh"

namespace claire {

namespace {
// ---------------------------------------------------------------- pass 1 ---
// x3 forward real -> half spectrum.  Block: L complex lines = 2L real lines.
template <int N, int L, typename TI = float>
__global__ void __launch_bounds__(kThreads)
k_r2c_x3(const TI *__restrict__ in, float2 *__restrict__ out, long long nlines, FftPlan p,
         int h3, int p3) {
    extern __shared__ float2 sm[];
    const int n = Fft<N>::size(p), ls = L + 1;
    float2 *A = sm, *B = sm + n * ls;
    const long long line0 = (long long)blockIdx.x * 2 * L;
    // real lines 2l and 2l+1 become the real and imaginary part of line l
        for (int t = threadIdx.x; t < L * n; t += blockDim.x) {
        const int l = t / n, e = t - l * n;
        const long long la = line0 + 2 * l;
        const float re = la < nlines ? ldr(in + la * n + e) : 0.f;
        const float im = la + 1 < nlines ? ldr(in + (la + 1) * n + e) : 0.f;
        A[e * ls + l] = make_float2(re, im);
    }
    __syncthreads();
    float2 *Rz = Fft<N>::template run<L>(A, B, p, ls, -1.f);
    if (N > 0) h3 = N / 2 + 1;
    for (int t = threadIdx.x; t < L * h3; t += blockDim.x) {
        const int l = t / h3, k = t - l * h3;
        const float2 z = Rz[k * ls + l];
        const float2 zn = Rz[((k == 0) ? 0 : (n - k)) * ls + l];
        // A_k = (Z_k + conj Z_{n-k})/2,  B_k = -i (Z_k - conj Z_{n-k})/2
        const float2 a = make_float2(0.5f * (z.x + zn.x), 0.5f * (z.y - zn.y));
        const float2 b = make_float2(0.5f * (z.y + zn.y), -0.5f * (z.x - zn.x));
        const long long la = line0 + 2 * l;
        if (la < nlines) out[la * p3 + k] = a;
        if (la + 1 < nlines) out[(la + 1) * p3 + k] = b;
    }
}

// Pass 1 with persistent blocks: the 2L real lines of the next tile (one
// contiguous chunk) are fetched by 16-byte cp.async into a staging buffer
// while the current tile is transformed, then transposed into the transform
// layout.  FP32 input, n a multiple of 4, 16-byte aligned (the launcher
// checks; otherwise the one-tile-per-block form above runs).
template <int N, int L>
__global__ void __launch_bounds__(kThreads, fft_in_place(N) ? 3 : 1)
k_r2c_x3_p(const float *__restrict__ in, float2 *__restrict__ out, long long nlines, FftPlan p, int h3, int p3,
           int nitems) {
    extern __shared__ float2 sm[];
    constexpr bool IP = fft_in_place(N);  // in-place transform: no scratch tile
    const int n = Fft<N>::size(p), ls = L + 1;
    float2 *A = sm, *B = sm + n * ls;
    float *S = reinterpret_cast<float *>(sm + (IP ? 1 : 2) * n * ls);
    auto load = [&](int item) {
        const long long line0 = (long long)item * 2 * L;
        const float *base = in + line0 * n;
        const int nch = (2 * L * n) / 4;
        for (int t = threadIdx.x; t < nch; t += blockDim.x) {
            const long long line = line0 + (4 * t) / n;
            const int bytes = line < nlines ? 16 : 0;
            cp_async16z(S + 4 * t, base + (bytes ? 4 * t : 0), bytes);
        }
        cp_async_commit_all();
    };
    const int i0 = blockIdx.x, stride = gridDim.x;
    if (i0 >= nitems) return;
    load(i0);
    if (N > 0) h3 = N / 2 + 1;
    for (int item = i0; item < nitems; item += stride) {
        cp_async_wait_n<0>();
        __syncthreads();
        // real lines 2l and 2l+1 become the real and imaginary part of line l
        for (int t = threadIdx.x; t < L * n; t += blockDim.x) {
            const int l = t / n, e = t - l * n;
            A[e * ls + l] = make_float2(S[(2 * l) * n + e], S[(2 * l + 1) * n + e]);
        }
        __syncthreads();
        if (item + stride < nitems) load(item + stride);
        float2 *Rz = A;
        if constexpr (IP) fft_ip<N, L, kThreads, L + 1>(A, p.tw, -1.f);
        else Rz = Fft<N>::template run<L>(A, B, p, ls, -1.f);
        const long long line0 = (long long)item * 2 * L;
        for (int t = threadIdx.x; t < L * h3; t += blockDim.x) {
            const int l = t / h3, k = t - l * h3;
            const float2 z = Rz[k * ls + l];
            const float2 zn = Rz[((k == 0) ? 0 : (n - k)) * ls + l];
            const float2 a = make_float2(0.5f * (z.x + zn.x), 0.5f * (z.y - zn.y));
            const float2 b = make_float2(0.5f * (z.y + zn.y), -0.5f * (z.x - zn.x));
            const long long la = line0 + 2 * l;
            if (la < nlines) out[la * p3 + k] = a;
            if (la + 1 < nlines) out[(la + 1) * p3 + k] = b;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- pass 2 ---
// x2 complex transform in place.  Persistent blocks walk the tiles (TK k3
// columns of one (c, i1) plane) and double-buffer them: cp.async fetches the
// next tile while the current one is transformed (measured at 256^3: the x2
// passes of a solve 3.09 -> 2.44 ms against one tile per block).
template <int N, int TK>
__global__ void __launch_bounds__(kThreads)
k_c2c_x2(float2 *__restrict__ data, FftPlan p, int h3, int p3, float s, int ntk, int nitems) {
    extern __shared__ float2 sm[];
    const int n = Fft<N>::size(p);
    float2 *A0 = sm, *A1 = sm + n * TK, *B = sm + 2 * n * TK;
    auto load = [&](int item, float2 *dst) {
        const int plane = item / ntk, k0 = (item - plane * ntk) * TK;
        const float2 *base = data + (long long)plane * n * p3 + k0;
        for (int t = threadIdx.x; t < n * (TK / 2); t += blockDim.x) {
            const int e = t / (TK / 2), ch = t - e * (TK / 2);
            const int col = k0 + 2 * ch;
            const int bytes = col + 2 <= h3 ? 16 : (col < h3 ? 8 : 0);
            const float2 *src = base + (long long)e * p3 + (bytes ? 2 * ch : 0);
            cp_async16z(dst + e * TK + 2 * ch, src, bytes);
        }
        cp_async_commit_all();
    };
    const int i0 = blockIdx.x, stride = gridDim.x;
    if (i0 >= nitems) return;
    load(i0, A0);
    bool cur0 = true;
    for (int item = i0; item < nitems; item += stride) {
        float2 *Acur = cur0 ? A0 : A1, *Anext = cur0 ? A1 : A0;
        if (item + stride < nitems) {
            load(item + stride, Anext);
            cp_async_wait_n<1>();
        } else {
            cp_async_wait_n<0>();
        }
        __syncthreads();
        float2 *R = Fft<N>::template run<TK>(Acur, B, p, TK, s);
        const int plane = item / ntk, k0 = (item - plane * ntk) * TK;
        float2 *base = data + (long long)plane * n * p3 + k0;
        for (int t = threadIdx.x; t < n * TK; t += blockDim.x) {
            const int e = t / TK, l = t - e * TK;
            if (k0 + l < h3) base[(long long)e * p3 + l] = R[e * TK + l];
        }
        __syncthreads();
        cur0 = !cur0;
    }
}

// Pass 2 for lengths with an in-place compile-time plan (stage_ip): the
// transform needs no scratch tile, so a block holds only the current and the
// next tile (three blocks per SM at n2 = 256), and stores two columns
// (16 bytes) at a time.
template <int N, int TK, int MT, int MINB>
__global__ void __launch_bounds__(MT, MINB)
k_c2c_x2_ip(float2 *__restrict__ data, FftPlan p, int h3, int p3, float s, int ntk, int nitems) {
    extern __shared__ float2 sm[];
    constexpr int CH = TK / 2;  // 16-byte chunks per row
    float2 *cur = sm, *nxt = sm + N * TK;
    const float2 *__restrict__ tw = p.tw;
    auto load = [&](int item, float2 *dst) {
        const int plane = item / ntk, k0 = (item - plane * ntk) * TK;
        const float2 *base = data + (long long)plane * N * p3 + k0;
        for (int t = threadIdx.x; t < N * CH; t += MT) {
            const int e = t / CH, ch = t - e * CH;
            const int col = k0 + 2 * ch;
            const int bytes = col + 2 <= h3 ? 16 : (col < h3 ? 8 : 0);
            cp_async16z(dst + e * TK + 2 * ch, base + (long long)e * p3 + (bytes ? 2 * ch : 0), bytes);
        }
        cp_async_commit_all();
    };
    const int i0 = blockIdx.x, stride = gridDim.x;
    if (i0 >= nitems) return;
    load(i0, cur);
    for (int item = i0; item < nitems; item += stride) {
        if (item + stride < nitems) {
            load(item + stride, nxt);
            cp_async_wait_n<1>();
        } else {
            cp_async_wait_n<0>();
        }
        __syncthreads();
        fft_ip<N, TK, MT>(cur, tw, s);
        const int plane = item / ntk, k0 = (item - plane * ntk) * TK;
        float2 *base = data + (long long)plane * N * p3 + k0;
        for (int t = threadIdx.x; t < N * CH; t += MT) {
            const int e = t / CH, ch = t - e * CH;
            const int col = k0 + 2 * ch;
            // one 16-byte shared load per two columns (two 8-byte loads at a
            // 16-byte lane stride would conflict in pairs of banks)
            const float4 q = *reinterpret_cast<const float4 *>(cur + e * TK + 2 * ch);
            float2 *g = base + (long long)e * p3 + 2 * ch;
            if (col + 2 <= h3) *reinterpret_cast<float4 *>(g) = q;
            else if (col < h3) *g = make_float2(q.x, q.y);
        }
        __syncthreads();
        float2 *t = cur;
        cur = nxt;
        nxt = t;
    }
}

// ---------------------------------------------------------------- pass 3 ---
// The x1 pass's pointwise step at wavenumber (k1, k2, k3) for the three
// components a, b, c of one spectral point (kd = the wavenumber with an even
// axis's Nyquist index set to 0, used in the divergence penalty):
//   OP_A     beta |k|^2 I + gamma kd kd^T
//   OP_AINV  its inverse by Sherman-Morrison (identity at k = 0)
//   OP_X1INV scale only; OP_X1FWD nothing
// each times scale (the 1/N of the inverse transform).
template <int OP>
__device__ __forceinline__ void mul_point(float2 &pa, float2 &pb, float2 &pc, float k1, float k1d, float k2,
                                          float k2d, float k3, float k3d, const SpecParams &sp) {
    if (OP == OP_X1FWD) {
    } else if (OP == OP_X1INV) {
        pa = make_float2(pa.x * sp.scale, pa.y * sp.scale);
        pb = make_float2(pb.x * sp.scale, pb.y * sp.scale);
        pc = make_float2(pc.x * sp.scale, pc.y * sp.scale);
    } else {
        const float2 a = pa, b = pb, c = pc;
        const float kk = k1 * k1 + k2 * k2 + k3 * k3;
        const float kd2 = k1d * k1d + k2d * k2d + k3d * k3d;
        const float2 kv = make_float2(k1d * a.x + k2d * b.x + k3d * c.x,
                                      k1d * a.y + k2d * b.y + k3d * c.y);
        float diag, coup;
        if (OP == OP_A) {
            diag = sp.beta * kk;
            coup = sp.gamma;
        } else {
            if (kk == 0.f) {
                diag = 1.f;
                coup = 0.f;
            } else {
                const float bk = sp.beta * kk;
                diag = 1.f / bk;
                coup = -sp.gamma * diag / (bk + sp.gamma * kd2);
            }
        }
        const float s = sp.scale;
        pa = make_float2((diag * a.x + coup * k1d * kv.x) * s, (diag * a.y + coup * k1d * kv.y) * s);
        pb = make_float2((diag * b.x + coup * k2d * kv.x) * s, (diag * b.y + coup * k2d * kv.y) * s);
        pc = make_float2((diag * c.x + coup * k3d * kv.x) * s, (diag * c.y + coup * k3d * kv.y) * s);
    }
}

// x1 forward, multiplier, x1 inverse, in place; all three components at once
// (the divergence penalty couples them).  Persistent blocks walk the items
// (TK k3 columns at one k2 index); the three component tiles of the next item
// are fetched by 16-byte cp.async (zero-filled past h3) while the current
// item is transformed, multiplied and transformed back.  Seven tiles of n1*TK:
// three current, three next, one scratch.
template <int N, int TK, int OP>
__global__ void __launch_bounds__(kThreads)
k_mul_x1(float2 *__restrict__ data, FftPlan p1, int n2, int n3, int h3, int p3, long long cstride, SpecParams sp,
           int ntk, int nitems) {
    constexpr bool FWD = OP != OP_X1INV, INV = OP != OP_X1FWD;
    extern __shared__ float2 sm[];
    const int n1 = Fft<N>::size(p1);
    const int tile = n1 * TK;
    float2 *cur[3] = {sm, sm + tile, sm + 2 * tile};
    float2 *scratch = sm + 3 * tile;
    float2 *nxt[3] = {sm + 4 * tile, sm + 5 * tile, sm + 6 * tile};
    const long long rowstride = (long long)n2 * p3;  // between consecutive i1
    constexpr int CH = TK / 2;                        // 16-byte chunks per row
    auto load = [&](int item, float2 *const *dst) {
        const int i2 = item / ntk, k0 = (item - i2 * ntk) * TK;
        const float2 *base = data + (long long)i2 * p3 + k0;
        for (int t = threadIdx.x; t < 3 * n1 * CH; t += blockDim.x) {
            const int c = t / (n1 * CH), r = t - c * n1 * CH;
            const int e = r / CH, ch = r - e * CH;
            const int col = k0 + 2 * ch;
            const int bytes = col + 2 <= h3 ? 16 : (col < h3 ? 8 : 0);
            cp_async16z(dst[c] + e * TK + 2 * ch, base + c * cstride + e * rowstride + (bytes ? 2 * ch : 0), bytes);
        }
        cp_async_commit_all();
    };
    const int i0 = blockIdx.x, stride = gridDim.x;
    if (i0 >= nitems) return;
    load(i0, cur);
    for (int item = i0; item < nitems; item += stride) {
        if (item + stride < nitems) {
            load(item + stride, nxt);
            cp_async_wait_n<1>();
        } else {
            cp_async_wait_n<0>();
        }
        __syncthreads();
        if (FWD) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float2 *r = Fft<N>::template run<TK>(cur[c], scratch, p1, TK, -1.f);
                if (r != cur[c]) { scratch = cur[c]; cur[c] = r; }
            }
        }
        const int i2 = item / ntk, k0 = (item - i2 * ntk) * TK;
        // multiplier at (k1, k2, k3)
        const float k2 = wavenumber(i2, n2), k2d = wavenumber_d1(i2, n2);
        for (int t = threadIdx.x; t < tile; t += blockDim.x) {
            const int e = t / TK, l = t - e * TK;
            const int i3 = k0 + l;
            const float k1 = wavenumber(e, n1), k1d = wavenumber_d1(e, n1);
            const float k3 = (float)i3, k3d = ((n3 & 1) == 0 && 2 * i3 == n3) ? 0.f : k3;
            const int id = e * TK + l;
            mul_point<OP>(cur[0][id], cur[1][id], cur[2][id], k1, k1d, k2, k2d, k3, k3d, sp);
        }
        __syncthreads();
        if (INV) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float2 *r = Fft<N>::template run<TK>(cur[c], scratch, p1, TK, +1.f);
                if (r != cur[c]) { scratch = cur[c]; cur[c] = r; }
            }
        }
        float2 *base = data + (long long)i2 * p3 + k0;
        for (int c = 0; c < 3; ++c) {
            for (int t = threadIdx.x; t < tile; t += blockDim.x) {
                const int e = t / TK, l = t - e * TK;
                if (k0 + l < h3) base[c * cstride + e * rowstride + l] = cur[c][e * TK + l];
            }
        }
        __syncthreads();
        // the next item's tiles become the current ones; the current tiles
        // (and the scratch the transforms left) are free again
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float2 *t = cur[c];
            cur[c] = nxt[c];
            nxt[c] = t;
        }
    }
}

// The same pass for lengths with a compile-time plan.  The three component
// tiles of an item are interleaved line by line -- 3 TK lines of n1 elements,
// buf[e * 3TK + c * TK + l] -- and transformed together, in place, by MT
// threads (stage_ip): one barrier pair per radix stage serves all three
// components, every thread holds a butterfly in every stage (at n1 = 256,
// TK = 8: 16 x 24 = 384 radix-16 butterflies for 384 threads), and no
// scratch tile is needed.  Six tiles of n1*TK: current and next item.
template <int N, int TK, int OP, int MT, int MINB>
__global__ void __launch_bounds__(MT, MINB)
k_mul_x1_ip(float2 *__restrict__ data, FftPlan p1, int n2, int n3, int h3, int p3, long long cstride,
            SpecParams sp, int ntk, int nitems) {
    constexpr bool FWD = OP != OP_X1INV, INV = OP != OP_X1FWD;
    constexpr int LL = 3 * TK, TILE = N * LL, CH = TK / 2;  // CH: 16-byte chunks per row and component
    extern __shared__ float2 sm[];
    float2 *cur = sm, *nxt = sm + TILE;
    const long long rowstride = (long long)n2 * p3;  // between consecutive i1
    const float2 *__restrict__ tw = p1.tw;
    auto load = [&](int item, float2 *dst) {
        const int i2 = item / ntk, k0 = (item - i2 * ntk) * TK;
        const float2 *base = data + (long long)i2 * p3 + k0;
        for (int t = threadIdx.x; t < 3 * N * CH; t += MT) {
            const int c = t / (N * CH), r = t - c * (N * CH);
            const int e = r / CH, ch = r - e * CH;
            const int col = k0 + 2 * ch;
            const int bytes = col + 2 <= h3 ? 16 : (col < h3 ? 8 : 0);
            cp_async16z(dst + e * LL + c * TK + 2 * ch, base + c * cstride + e * rowstride + (bytes ? 2 * ch : 0),
                        bytes);
        }
        cp_async_commit_all();
    };
    const int i0 = blockIdx.x, stride = gridDim.x;
    if (i0 >= nitems) return;
    load(i0, cur);
    for (int item = i0; item < nitems; item += stride) {
        if (item + stride < nitems) {
            load(item + stride, nxt);
            cp_async_wait_n<1>();
        } else {
            cp_async_wait_n<0>();
        }
        __syncthreads();
        if (FWD) fft_ip<N, LL, MT>(cur, tw, -1.f);
        const int i2 = item / ntk, k0 = (item - i2 * ntk) * TK;
        const float k2 = wavenumber(i2, n2), k2d = wavenumber_d1(i2, n2);
        for (int t = threadIdx.x; t < N * TK; t += MT) {
            const int e = t / TK, l = t - e * TK;
            const int i3 = k0 + l;
            const float k1 = wavenumber(e, N), k1d = wavenumber_d1(e, N);
            const float k3 = (float)i3, k3d = ((n3 & 1) == 0 && 2 * i3 == n3) ? 0.f : k3;
            float2 *q = cur + e * LL + l;
            mul_point<OP>(q[0], q[TK], q[2 * TK], k1, k1d, k2, k2d, k3, k3d, sp);
        }
        __syncthreads();
        if (INV) fft_ip<N, LL, MT>(cur, tw, +1.f);
        // back to global memory, two columns (16 bytes) per store
        float2 *base = data + (long long)i2 * p3 + k0;
        for (int t = threadIdx.x; t < 3 * N * CH; t += MT) {
            const int c = t / (N * CH), r = t - c * (N * CH);
            const int e = r / CH, ch = r - e * CH;
            const int col = k0 + 2 * ch;
            const float4 q = *reinterpret_cast<const float4 *>(cur + e * LL + c * TK + 2 * ch);
            float2 *g = base + c * cstride + e * rowstride + 2 * ch;
            if (col + 2 <= h3) *reinterpret_cast<float4 *>(g) = q;
            else if (col < h3) *g = make_float2(q.x, q.y);
        }
        __syncthreads();
        float2 *t = cur;
        cur = nxt;
        nxt = t;
    }
}

// ---------------------------------------------------------------- pass 5 ---
// x3 inverse half spectrum -> real, two real lines per complex transform.
template <int N, int L, int EPI, typename TO = float>
__global__ void __launch_bounds__(kThreads)
k_c2r_x3(const float2 *__restrict__ in, TO *__restrict__ out, const float *__restrict__ add,
         long long nlines, FftPlan p, int h3, int p3) {
    extern __shared__ float2 sm[];
    const int n = Fft<N>::size(p), ls = L + 1;
    float2 *A = sm, *B = sm + n * ls;
    const long long line0 = (long long)blockIdx.x * 2 * L;
    const bool even = (n & 1) == 0;
#pragma unroll
    for (int t = threadIdx.x; t < L * n; t += kThreads) {
        const int l = t / n, k = t - l * n;
        const long long la = line0 + 2 * l;
        const bool lo = k < h3;
        const int kk = lo ? k : n - k;
        float2 a = la < nlines ? in[la * p3 + kk] : make_float2(0.f, 0.f);
        float2 b = la + 1 < nlines ? in[(la + 1) * p3 + kk] : make_float2(0.f, 0.f);
        if (k == 0 || (even && 2 * k == n)) {
            a.y = 0.f;
            b.y = 0.f;
        }
        if (!lo) {
            a.y = -a.y;
            b.y = -b.y;
        }
        // Z = A + i B
        A[k * ls + l] = make_float2(a.x - b.y, a.y + b.x);
    }
    __syncthreads();
    float2 *R = Fft<N>::template run<L>(A, B, p, ls, +1.f);
    for (int t = threadIdx.x; t < L * n; t += blockDim.x) {
        const int l = t / n, e = t - l * n;
        const long long la = line0 + 2 * l;
        const float2 z = R[e * ls + l];
        if (la < nlines) {
            float val = z.x;
            if (EPI == EPI_ADD) val += add[la * n + e];
            str(out + la * n + e, val);
        }
        if (la + 1 < nlines) {
            float val = z.y;
            if (EPI == EPI_ADD) val += add[(la + 1) * n + e];
            str(out + (la + 1) * n + e, val);
        }
    }
}

// Pass 5 with persistent blocks: the 2L half-spectrum lines of the next tile
// (one contiguous chunk of 2L*p3 complex values) are fetched by 16-byte
// cp.async into a staging buffer while the current tile is transformed.
template <int N, int L, int EPI, typename TO = float>
__global__ void __launch_bounds__(kThreads, fft_in_place(N) ? 3 : 1)
k_c2r_x3_p(const float2 *__restrict__ in, TO *__restrict__ out, const float *__restrict__ add, long long nlines,
           FftPlan p, int h3, int p3, int nitems) {
    extern __shared__ float2 sm[];
    constexpr bool IP = fft_in_place(N);  // in-place transform: no scratch tile
    const int n = Fft<N>::size(p), ls = L + 1;
    float2 *A = sm, *B = sm + n * ls;
    float2 *S = sm + (IP ? 1 : 2) * n * ls;  // staging: 2L lines of p3 complex values
    const bool even = (n & 1) == 0;
    if (N > 0) h3 = N / 2 + 1;
    auto load = [&](int item) {
        const long long line0 = (long long)item * 2 * L;
        const float2 *base = in + line0 * p3;
        const int nch = L * p3;  // 2L * p3 complex values, two per chunk
        for (int t = threadIdx.x; t < nch; t += blockDim.x) {
            const long long line = line0 + (2 * t) / p3;
            const int bytes = line < nlines ? 16 : 0;
            cp_async16z(S + 2 * t, base + (bytes ? 2 * t : 0), bytes);
        }
        cp_async_commit_all();
    };
    const int i0 = blockIdx.x, stride = gridDim.x;
    if (i0 >= nitems) return;
    load(i0);
    for (int item = i0; item < nitems; item += stride) {
        cp_async_wait_n<0>();
        __syncthreads();
        // each stored coefficient k < h3 gives Z_k = A_k + i B_k and, by
        // Hermitian symmetry, Z_{n-k} = conj(A_k) + i conj(B_k): one read of
        // the staged lines for both
        for (int t = threadIdx.x; t < L * h3; t += blockDim.x) {
            const int l = t / h3, k = t - l * h3;
            float2 a = S[(2 * l) * p3 + k];
            float2 b = S[(2 * l + 1) * p3 + k];
            const bool self = k == 0 || (even && 2 * k == n);
            if (self) {
                a.y = 0.f;
                b.y = 0.f;
            }
            A[k * ls + l] = make_float2(a.x - b.y, a.y + b.x);
            if (!self) A[(n - k) * ls + l] = make_float2(a.x + b.y, -a.y + b.x);
        }
        __syncthreads();
        if (item + stride < nitems) load(item + stride);
        float2 *R = A;
        if constexpr (IP) fft_ip<N, L, kThreads, L + 1>(A, p.tw, +1.f);
        else R = Fft<N>::template run<L>(A, B, p, ls, +1.f);
        const long long line0 = (long long)item * 2 * L;
        for (int t = threadIdx.x; t < L * n; t += blockDim.x) {
            const int l = t / n, e = t - l * n;
            const long long la = line0 + 2 * l;
            const float2 z = R[e * ls + l];
            if (la < nlines) {
                float val = z.x;
                if (EPI == EPI_ADD) val += add[la * n + e];
                str(out + la * n + e, val);
            }
            if (la + 1 < nlines) {
                float val = z.y;
                if (EPI == EPI_ADD) val += add[(la + 1) * n + e];
                str(out + (la + 1) * n + e, val);
            }
        }
        __syncthreads();
    }
}

// -------------------------------------------------------------- launchers --
}  // namespace

int persistent_grid(long long nitems, size_t smem) {
    static int sms[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    if (!sms[dev]) {
        int c = 0;
        if (cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c <= 0) c = 152;
        sms[dev] = c;
    }
    long long per_sm = (long long)(227 * 1024) / (long long)(smem + 1024);
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 8) per_sm = 8;
    const long long g = per_sm * sms[dev];
    return (int)(nitems < g ? nitems : g);
}

namespace {

template <int N, int L, typename TI>
void r2c_l(const Dims &d, const FftPlan &p, const TI *in, float2 *out, long long nlines,
           cudaStream_t st) {
    if constexpr (std::is_same<TI, float>::value) {
        if (d.n3 % 4 == 0 && ((uintptr_t)in & 15) == 0) {
            const size_t smem = (fft_in_place(N) ? 1 : 2) * (size_t)d.n3 * (L + 1) * sizeof(float2) +
                                (size_t)2 * L * d.n3 * sizeof(float);
            const int nitems = (int)((nlines + 2 * L - 1) / (2 * L));
            set_smem<k_r2c_x3_p<N, L>>(smem);
            k_r2c_x3_p<N, L><<<persistent_grid(nitems, smem), kThreads, smem, st>>>(in, out, nlines, p, d.h3, d.p3,
                                                                                    nitems);
            return;
        }
    }
    const size_t smem = 2 * (size_t)d.n3 * (L + 1) * sizeof(float2);
    const long long blocks = (nlines + 2 * L - 1) / (2 * L);
    set_smem<k_r2c_x3<N, L, TI>>(smem);
    k_r2c_x3<N, L, TI><<<(unsigned)blocks, kThreads, smem, st>>>(in, out, nlines, p, d.h3, d.p3);
}

template <int N, typename TI>
void r2c_n(const Dims &d, const FftPlan &p, const TI *in, float2 *out, int ncomp,
           cudaStream_t st) {
    const long long nlines = (long long)ncomp * d.n1 * d.n2;
    if constexpr (N > 0) {
        r2c_l<N, lines_x3(N)>(d, p, in, out, nlines, st);
    } else {
        switch (lines_x3(d.n3)) {
            case 16: r2c_l<N, 16>(d, p, in, out, nlines, st); break;
            case 8: r2c_l<N, 8>(d, p, in, out, nlines, st); break;
            default: r2c_l<N, 4>(d, p, in, out, nlines, st); break;
        }
    }
}

template <typename TI>
void r2c_x3(const Dims &d, const FftPlan &p, const TI *in, float2 *out, int ncomp,
            cudaStream_t st) {
    switch (d.n3) {
#define CASE_N(NN) case NN: r2c_n<NN>(d, p, in, out, ncomp, st); return;
        CLAIRE_CT_SIZES(CASE_N)
#undef CASE_N
        default: r2c_n<0>(d, p, in, out, ncomp, st);
    }
}

template <int N, int TK>
void c2c_t(const Dims &d, const FftPlan &p, float2 *data, int ncomp, float s, cudaStream_t st) {
    const size_t smem = 3 * (size_t)d.n2 * TK * sizeof(float2);
    const int ntk = (d.h3 + TK - 1) / TK, nitems = ntk * ncomp * d.n1;
    const int grid = persistent_grid(nitems, smem);
    set_smem<k_c2c_x2<N, TK>>(smem);
    k_c2c_x2<N, TK><<<grid, kThreads, smem, st>>>(data, p, d.h3, d.p3, s, ntk, nitems);
}

template <int N, int TK>
void c2c_ip(const Dims &d, const FftPlan &p, float2 *data, int ncomp, float s, cudaStream_t st) {
    constexpr int MT = 256;
    constexpr size_t smem = 2 * (size_t)N * TK * sizeof(float2);
    constexpr int MINB = smem <= 72 * 1024 ? 3 : 2;
    const int ntk = (d.h3 + TK - 1) / TK, nitems = ntk * ncomp * d.n1;
    set_smem<k_c2c_x2_ip<N, TK, MT, MINB>>(smem);
    k_c2c_x2_ip<N, TK, MT, MINB><<<persistent_grid(nitems, smem), MT, smem, st>>>(data, p, d.h3, d.p3, s, ntk,
                                                                                  nitems);
}

template <int N>
void c2c_n(const Dims &d, const FftPlan &p, float2 *data, int ncomp, float s, cudaStream_t st) {
    if constexpr (fft_in_place(N)) {
        c2c_ip<N, tile_cols(N, 1)>(d, p, data, ncomp, s, st);
    } else if constexpr (N > 0) {
        c2c_t<N, tile_cols(N, 2)>(d, p, data, ncomp, s, st);
    } else {
        switch (tile_cols(d.n2, 2)) {
            case 16: c2c_t<N, 16>(d, p, data, ncomp, s, st); break;
            case 8: c2c_t<N, 8>(d, p, data, ncomp, s, st); break;
            default: c2c_t<N, 4>(d, p, data, ncomp, s, st); break;
        }
    }
}

void c2c_x2(const Dims &d, const FftPlan &p, float2 *data, int ncomp, float s, cudaStream_t st) {
    switch (d.n2) {
#define CASE_N(NN) case NN: c2c_n<NN>(d, p, data, ncomp, s, st); return;
        CLAIRE_CT_SIZES(CASE_N)
#undef CASE_N
        default: c2c_n<0>(d, p, data, ncomp, s, st);
    }
}

template <int N, int TK, int OP>
void mul_t(const Dims &d, const FftPlan &p, float2 *data, const SpecParams &sp, cudaStream_t st) {
    const size_t smem = (size_t)7 * d.n1 * TK * sizeof(float2);
    const long long cstride = (long long)d.n1 * d.n2 * d.p3;
    const int ntk = (d.h3 + TK - 1) / TK, nitems = ntk * d.n2;
    set_smem<k_mul_x1<N, TK, OP>>(smem);
    k_mul_x1<N, TK, OP><<<persistent_grid(nitems, smem), kThreads, smem, st>>>(data, p, d.n2, d.n3, d.h3, d.p3,
                                                                                cstride, sp, ntk, nitems);
}

// compile-time plans: the interleaved in-place form, 384 threads, six tiles
template <int N, int TK, int OP>
void mul_ip(const Dims &d, const FftPlan &p, float2 *data, const SpecParams &sp, cudaStream_t st) {
    constexpr int MT = 384;
    constexpr size_t smem = (size_t)6 * N * TK * sizeof(float2);
    constexpr int MINB = smem <= 112 * 1024 ? 2 : 1;
    const long long cstride = (long long)d.n1 * d.n2 * d.p3;
    const int ntk = (d.h3 + TK - 1) / TK, nitems = ntk * d.n2;
    set_smem<k_mul_x1_ip<N, TK, OP, MT, MINB>>(smem);
    k_mul_x1_ip<N, TK, OP, MT, MINB><<<persistent_grid(nitems, smem), MT, smem, st>>>(data, p, d.n2, d.n3, d.h3,
                                                                                       d.p3, cstride, sp, ntk, nitems);
}

template <int N, int OP>
void mul_n(const Dims &d, const FftPlan &p, float2 *data, const SpecParams &sp, cudaStream_t st) {
    constexpr int NB = 6;  // three component tiles for the current item, three for the next
    if constexpr (fft_in_place(N)) {
        // six tiles in all (no scratch): the column count of five data tiles and one more
        mul_ip<N, tile_cols(N, NB - 1), OP>(d, p, data, sp, st);
    } else if constexpr (N > 0) {
        mul_t<N, tile_cols(N, NB), OP>(d, p, data, sp, st);
    } else {
        switch (tile_cols(d.n1, NB)) {
            case 16: mul_t<N, 16, OP>(d, p, data, sp, st); break;
            case 8: mul_t<N, 8, OP>(d, p, data, sp, st); break;
            default: mul_t<N, 4, OP>(d, p, data, sp, st); break;
        }
    }
}

template <int OP>
void mul_x1_op(const Dims &d, const FftPlan &p, float2 *data, const SpecParams &sp,
               cudaStream_t st) {
    switch (d.n1) {
#define CASE_N(NN) case NN: mul_n<NN, OP>(d, p, data, sp, st); return;
        CLAIRE_CT_SIZES(CASE_N)
#undef CASE_N
        default: mul_n<0, OP>(d, p, data, sp, st);
    }
}

template <int N, int L, typename TO>
void c2r_l(const Dims &d, const FftPlan &p, const float2 *in, TO *out, const float *add,
           long long nlines, cudaStream_t st) {
    if (((uintptr_t)in & 15) == 0) {
        // the persistent form with the next tile staged by cp.async
        const size_t smem = (fft_in_place(N) ? 1 : 2) * (size_t)d.n3 * (L + 1) * sizeof(float2) +
                            (size_t)2 * L * d.p3 * sizeof(float2);
        const int nitems = (int)((nlines + 2 * L - 1) / (2 * L));
        const int grid = persistent_grid(nitems, smem);
        if (add) {
            set_smem<k_c2r_x3_p<N, L, EPI_ADD, TO>>(smem);
            k_c2r_x3_p<N, L, EPI_ADD, TO><<<grid, kThreads, smem, st>>>(in, out, add, nlines, p, d.h3, d.p3, nitems);
        } else {
            set_smem<k_c2r_x3_p<N, L, EPI_STORE, TO>>(smem);
            k_c2r_x3_p<N, L, EPI_STORE, TO><<<grid, kThreads, smem, st>>>(in, out, add, nlines, p, d.h3, d.p3,
                                                                          nitems);
        }
        return;
    }
    const size_t smem = 2 * (size_t)d.n3 * (L + 1) * sizeof(float2);
    const long long blocks = (nlines + 2 * L - 1) / (2 * L);
    if (add) {
        set_smem<k_c2r_x3<N, L, EPI_ADD, TO>>(smem);
        k_c2r_x3<N, L, EPI_ADD, TO><<<(unsigned)blocks, kThreads, smem, st>>>(in, out, add, nlines, p,
                                                                              d.h3, d.p3);
    } else {
        set_smem<k_c2r_x3<N, L, EPI_STORE, TO>>(smem);
        k_c2r_x3<N, L, EPI_STORE, TO><<<(unsigned)blocks, kThreads, smem, st>>>(in, out, add, nlines,
                                                                                p, d.h3, d.p3);
    }
}

template <int N, typename TO>
void c2r_n(const Dims &d, const FftPlan &p, const float2 *in, TO *out, const float *add,
           int ncomp, cudaStream_t st) {
    const long long nlines = (long long)ncomp * d.n1 * d.n2;
    if constexpr (N > 0) {
        c2r_l<N, lines_x3(N)>(d, p, in, out, add, nlines, st);
    } else {
        switch (lines_x3(d.n3)) {
            case 16: c2r_l<N, 16>(d, p, in, out, add, nlines, st); break;
            case 8: c2r_l<N, 8>(d, p, in, out, add, nlines, st); break;
            default: c2r_l<N, 4>(d, p, in, out, add, nlines, st); break;
        }
    }
}

template <typename TO>
void c2r_x3(const Dims &d, const FftPlan &p, const float2 *in, TO *out, const float *add,
            int ncomp, cudaStream_t st) {
    switch (d.n3) {
#define CASE_N(NN) case NN: c2r_n<NN>(d, p, in, out, add, ncomp, st); return;
        CLAIRE_CT_SIZES(CASE_N)
#undef CASE_N
        default: c2r_n<0>(d, p, in, out, add, ncomp, st);
    }
}

// ------------------------------------------------------ grid resampling ---
__device__ __forceinline__ bool in_coarse_band(float k, int nc) { return 2.f * fabsf(k) < (float)nc; }
__device__ __forceinline__ int index_of(float k, int n) { return k < 0.f ? n + (int)k : (int)k; }

// thread per coarse (component, i1, i2, k3)
__global__ void k_spec_restrict(const float2 *__restrict__ sf, Dims df, float2 *__restrict__ sc,
                                Dims dc, float scale) {
    const long long per_c = (long long)dc.n1 * dc.n2 * dc.h3;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= 3 * per_c) return;
    const int c = (int)(t / per_c);
    long long r = t - c * per_c;
    const int k3 = (int)(r % dc.h3);
    r /= dc.h3;
    const int i2 = (int)(r % dc.n2), i1 = (int)(r / dc.n2);
    const float k1 = wavenumber(i1, dc.n1), k2 = wavenumber(i2, dc.n2);
    float2 v = make_float2(0.f, 0.f);
    if (in_coarse_band(k1, dc.n1) && in_coarse_band(k2, dc.n2) && in_coarse_band((float)k3, dc.n3)) {
        const long long src = (((long long)c * df.n1 + index_of(k1, df.n1)) * df.n2 + index_of(k2, df.n2)) *
                              df.p3 + k3;
        const float2 f = sf[src];
        v = make_float2(f.x * scale, f.y * scale);
    }
    sc[(((long long)c * dc.n1 + i1) * dc.n2 + i2) * dc.p3 + k3] = v;
}

// thread per fine (i1, i2, k3), all three components (the inverse couples them)
__global__ void k_spec_twolevel(float2 *__restrict__ sf, Dims df, const float2 *__restrict__ sc,
                                Dims dc, float scale, float beta0, float gamma) {
    const long long per_c = (long long)df.n1 * df.n2 * df.h3;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= per_c) return;
    long long r = t;
    const int k3i = (int)(r % df.h3);
    r /= df.h3;
    const int i2 = (int)(r % df.n2), i1 = (int)(r / df.n2);
    const long long cs = (long long)df.n1 * df.n2 * df.p3;
    const long long id = ((long long)i1 * df.n2 + i2) * df.p3 + k3i;
    const float k1 = wavenumber(i1, df.n1), k2 = wavenumber(i2, df.n2), k3 = (float)k3i;
    if (in_coarse_band(k1, dc.n1) && in_coarse_band(k2, dc.n2) && in_coarse_band(k3, dc.n3)) {
        const long long ccs = (long long)dc.n1 * dc.n2 * dc.p3;
        const long long src = ((long long)index_of(k1, dc.n1) * dc.n2 + index_of(k2, dc.n2)) * dc.p3 + k3i;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float2 f = sc[c * ccs + src];
            sf[c * cs + id] = make_float2(f.x * scale, f.y * scale);
        }
    } else {
        // (beta0 A)^{-1} by Sherman-Morrison (never k = 0 here)
        const float k1d = wavenumber_d1(i1, df.n1), k2d = wavenumber_d1(i2, df.n2);
        const float k3d = ((df.n3 & 1) == 0 && 2 * k3i == df.n3) ? 0.f : k3;
        const float kk = k1 * k1 + k2 * k2 + k3 * k3, kd2 = k1d * k1d + k2d * k2d + k3d * k3d;
        const float bk = beta0 * kk, diag = 1.f / bk, coup = -gamma * diag / (bk + gamma * kd2);
        const float2 a = sf[id], b = sf[cs + id], c = sf[2 * cs + id];
        const float2 kv = make_float2(k1d * a.x + k2d * b.x + k3d * c.x, k1d * a.y + k2d * b.y + k3d * c.y);
        sf[id] = make_float2(diag * a.x + coup * k1d * kv.x, diag * a.y + coup * k1d * kv.y);
        sf[cs + id] = make_float2(diag * b.x + coup * k2d * kv.x, diag * b.y + coup * k2d * kv.y);
        sf[2 * cs + id] = make_float2(diag * c.x + coup * k3d * kv.x, diag * c.y + coup * k3d * kv.y);
    }
}

}  // namespace

void spectral_apply(const Dims &d, const FftPlan *ax, SpecOp op, const SpecParams &sp,
                    const float *in, float *out, const float *add, float2 *spec, cudaStream_t st,
                    Profiler *prof) {
    // first derivatives go through the axis transforms (fft_axis.cu); the
    // 3D passes below serve the operators that couple wavenumbers, A and A^-1
    if (op == OP_GRAD) {
        spectral_grad_1d(d, ax, in, out, st, prof);
        return;
    }
    if (op == OP_DIV) {
        spectral_div_1d(d, ax, in, out, st, prof);
        return;
    }
    const int nin = 3, nout = 3;
    // algorithmic bytes: real fields 4 B/voxel, half spectra 8 B per stored mode
    const double R = 4.0 * d.N, C = 8.0 * d.n1 * d.n2 * d.h3;
    {
        ProfScope ps(prof, CLAIRE_K_FFT_R2C, st, nin * (R + C));
        r2c_x3(d, ax[2], in, spec, nin, st);
    }
    {
        ProfScope ps(prof, CLAIRE_K_FFT_C2C, st, nin * 2 * C);
        c2c_x2(d, ax[1], spec, nin, -1.f, st);
    }
    {
        ProfScope ps(prof, CLAIRE_K_FFT_MUL, st, (nin + nout) * C);
        switch (op) {
            case OP_A: mul_x1_op<OP_A>(d, ax[0], spec, sp, st); break;
            case OP_AINV: mul_x1_op<OP_AINV>(d, ax[0], spec, sp, st); break;
            default: break;
        }
    }
    {
        ProfScope ps(prof, CLAIRE_K_FFT_C2C, st, nout * 2 * C);
        c2c_x2(d, ax[1], spec, nout, +1.f, st);
    }
    {
        ProfScope ps(prof, CLAIRE_K_FFT_C2R, st, nout * (R + C + (add ? R : 0.0)));
        c2r_x3(d, ax[2], spec, out, add, nout, st);
    }
}

}  // namespace claire

namespace claire {

void spectral_forward3(const Dims &d, const FftPlan *ax, const float *in, float2 *spec,
                       cudaStream_t st, Profiler *prof) {
    const double R = 4.0 * d.N, C = 8.0 * d.n1 * d.n2 * d.h3;
    {
        ProfScope ps(prof, CLAIRE_K_FFT_R2C, st, 3 * (R + C));
        r2c_x3(d, ax[2], in, spec, 3, st);
    }
    {
        ProfScope ps(prof, CLAIRE_K_FFT_C2C, st, 3 * 2 * C);
        c2c_x2(d, ax[1], spec, 3, -1.f, st);
    }
    {
        ProfScope ps(prof, CLAIRE_K_FFT_MUL, st, 6 * C);
        mul_x1_op<OP_X1FWD>(d, ax[0], spec, SpecParams{0.f, 0.f, 1.f}, st);
    }
}

void spectral_inverse3(const Dims &d, const FftPlan *ax, float2 *spec, float *out, float scale,
                       cudaStream_t st, Profiler *prof) {
    const double R = 4.0 * d.N, C = 8.0 * d.n1 * d.n2 * d.h3;
    {
        ProfScope ps(prof, CLAIRE_K_FFT_MUL, st, 6 * C);
        mul_x1_op<OP_X1INV>(d, ax[0], spec, SpecParams{0.f, 0.f, scale}, st);
    }
    {
        ProfScope ps(prof, CLAIRE_K_FFT_C2C, st, 3 * 2 * C);
        c2c_x2(d, ax[1], spec, 3, +1.f, st);
    }
    {
        ProfScope ps(prof, CLAIRE_K_FFT_C2R, st, 3 * (R + C));
        c2r_x3(d, ax[2], spec, out, nullptr, 3, st);
    }
}

void launch_spec_restrict(const Dims &df, const float2 *specf, const Dims &dc, float2 *specc,
                          float scale, cudaStream_t st, Profiler *prof) {
    const long long n = 3LL * dc.n1 * dc.n2 * dc.h3;
    ProfScope ps(prof, CLAIRE_K_FFT_MUL, st, 16.0 * n);
    k_spec_restrict<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(specf, df, specc, dc, scale);
}

void launch_spec_twolevel(const Dims &df, float2 *specf, const Dims &dc, const float2 *specc,
                          float scale, float beta0, float gamma, cudaStream_t st, Profiler *prof) {
    const long long n = (long long)df.n1 * df.n2 * df.h3;
    ProfScope ps(prof, CLAIRE_K_FFT_MUL, st, 48.0 * n);
    k_spec_twolevel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(specf, df, specc, dc, scale, beta0,
                                                                 gamma);
}

}  // namespace claire
