// fft_axis.cu -- spectral first derivatives by axis transforms (paper
// Section 3 "Discretization": first derivatives are spectral).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "claire_internal.cuh"
#include "fft_core.cuh"

namespace claire {

namespace {

// ------------------------------------------------------ axis derivatives ---
// The spectral first derivative along axis a only involves that axis:
// F^-1[i k^_a F f] = F_a^-1[i k^_a F_a f], because the multiplier depends on
// k_a alone and the 3D transform factorises into axis transforms (R4: k^_a is
// 0 at the Nyquist index of an even axis).  So d f/d x_a is one pass over f:
// load lines along x_a, transform, multiply by i k^_a / n_a, transform back,
// store.  Two real lines travel as the real and imaginary part of one complex
// line (the derivative kernel is real, so the parts stay apart).  A gradient
// is three such passes, a divergence three passes accumulating into one field:
// ~24 / 32 bytes per voxel instead of ~90 / ~80 through the 3D transform.

// real lines contiguous along x3; out (or out = add + ..., add may be out)
template <int N, int L, int EPI, typename TO>
__global__ void __launch_bounds__(kThreads)
k_deriv_x3(const float *__restrict__ in, TO *out, const float *add, long long nlines, FftPlan p) {
    extern __shared__ float2 sm[];
    const int n = Fft<N>::size(p), ls = L + 1;
    float2 *A = sm, *B = sm + n * ls;
    const long long line0 = (long long)blockIdx.x * 2 * L;
    for (int t = threadIdx.x; t < L * n; t += blockDim.x) {
        const int l = t / n, e = t - l * n;
        const long long la = line0 + 2 * l;
        const float re = la < nlines ? in[la * n + e] : 0.f;
        const float im = la + 1 < nlines ? in[(la + 1) * n + e] : 0.f;
        A[e * ls + l] = make_float2(re, im);
    }
    __syncthreads();
    float2 *R = Fft<N>::template run<L>(A, B, p, ls, -1.f);
    const float sc = 1.f / (float)n;
    for (int t = threadIdx.x; t < L * n; t += blockDim.x) {
        const int e = t / L, l = t - e * L;
        const float k = wavenumber_d1(e, n) * sc;
        const float2 z = R[e * ls + l];
        R[e * ls + l] = make_float2(-k * z.y, k * z.x);
    }
    __syncthreads();
    float2 *S = Fft<N>::template run<L>(R, R == A ? B : A, p, ls, +1.f);
    for (int t = threadIdx.x; t < L * n; t += blockDim.x) {
        const int l = t / n, e = t - l * n;
        const long long la = line0 + 2 * l;
        const float2 z = S[e * ls + l];
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

// The same pass with persistent blocks: the 2L real lines of the next tile
// (one contiguous chunk of 2L*n floats) are fetched by 16-byte cp.async into a
// staging buffer while the current tile is transformed; the tile is then
// transposed from the staging buffer into the transform layout.  Needs n a
// multiple of 4 and 16-byte aligned fields (the launcher checks).
template <int N, int L, int EPI, typename TO>
__global__ void __launch_bounds__(kThreads, fft_in_place(N) ? (N >= 256 ? 3 : 2) : 1)
k_deriv_x3_p(const float *__restrict__ in, TO *out, const float *add, long long nlines, FftPlan p, int nitems) {
    extern __shared__ float2 sm[];
    constexpr bool IP = fft_in_place(N);  // in-place transforms: no scratch tile
    const int n = Fft<N>::size(p), ls = L + 1;
    float2 *A = sm, *B = sm + n * ls;
    float *S = reinterpret_cast<float *>(sm + (IP ? 1 : 2) * n * ls);  // staging: 2L lines of n floats
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
    const float sc = 1.f / (float)n;
    for (int item = i0; item < nitems; item += stride) {
        cp_async_wait_n<0>();
        __syncthreads();
        for (int t = threadIdx.x; t < L * n; t += blockDim.x) {
            const int l = t / n, e = t - l * n;
            A[e * ls + l] = make_float2(S[(2 * l) * n + e], S[(2 * l + 1) * n + e]);
        }
        __syncthreads();
        if (item + stride < nitems) load(item + stride);
        float2 *R = A;
        if constexpr (IP) {
            // the multiplier i k / n applied as the last forward stage stores
            const auto deriv = [sc](int e, float2 &z) {
                const float k = wavenumber_d1(e, N) * sc;
                z = make_float2(-k * z.y, k * z.x);
            };
            fft_ip<N, L, kThreads, L + 1, 0>(A, p.tw, -1.f, deriv);
        } else {
            R = Fft<N>::template run<L>(A, B, p, ls, -1.f);
            for (int t = threadIdx.x; t < L * n; t += blockDim.x) {
                const int e = t / L, l = t - e * L;
                const float k = wavenumber_d1(e, n) * sc;
                const float2 z = R[e * ls + l];
                R[e * ls + l] = make_float2(-k * z.y, k * z.x);
            }
            __syncthreads();
        }
        float2 *Q = R;
        if constexpr (IP) fft_ip<N, L, kThreads, L + 1>(R, p.tw, +1.f);
        else Q = Fft<N>::template run<L>(R, R == A ? B : A, p, ls, +1.f);
        const long long line0 = (long long)item * 2 * L;
        for (int t = threadIdx.x; t < L * n; t += blockDim.x) {
            const int l = t / n, e = t - l * n;
            const long long la = line0 + 2 * l;
            const float2 z = Q[e * ls + l];
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

// lines along a strided axis (x2: element stride n3, planes i1; x1: element
// stride n2*n3, planes i2); a tile is 2*TKC consecutive x3 columns of one
// plane, adjacent columns paired into one complex column
template <int N, int TKC, int EPI, typename TO>
__global__ void __launch_bounds__(kThreads)
k_deriv_strided(const float *__restrict__ in, TO *out, const float *add, int n3, long long estride,
                long long pstride, FftPlan p) {
    extern __shared__ float2 sm[];
    const int n = Fft<N>::size(p);
    float2 *A = sm, *B = sm + n * TKC;
    const long long base = (long long)blockIdx.y * pstride;
    const int k0 = blockIdx.x * 2 * TKC;
    for (int t = threadIdx.x; t < n * TKC; t += blockDim.x) {
        const int e = t / TKC, c = t - e * TKC;
        const int i3 = k0 + 2 * c;
        const long long o = base + e * estride + i3;
        const float re = i3 < n3 ? in[o] : 0.f;
        const float im = i3 + 1 < n3 ? in[o + 1] : 0.f;
        A[e * TKC + c] = make_float2(re, im);
    }
    __syncthreads();
    float2 *R = Fft<N>::template run<TKC>(A, B, p, TKC, -1.f);
    const float sc = 1.f / (float)n;
    for (int t = threadIdx.x; t < n * TKC; t += blockDim.x) {
        const int e = t / TKC;
        const float k = wavenumber_d1(e, n) * sc;
        const float2 z = R[t];
        R[t] = make_float2(-k * z.y, k * z.x);
    }
    __syncthreads();
    float2 *S = Fft<N>::template run<TKC>(R, R == A ? B : A, p, TKC, +1.f);
    for (int t = threadIdx.x; t < n * TKC; t += blockDim.x) {
        const int e = t / TKC, c = t - e * TKC;
        const int i3 = k0 + 2 * c;
        const long long o = base + e * estride + i3;
        const float2 z = S[t];
        if (i3 < n3) {
            float val = z.x;
            if (EPI == EPI_ADD) val += add[o];
            str(out + o, val);
        }
        if (i3 + 1 < n3) {
            float val = z.y;
            if (EPI == EPI_ADD) val += add[o + 1];
            str(out + o + 1, val);
        }
    }
}

// The same pass with persistent blocks that double-buffer their tiles: cp.async
// fetches the next tile (2*TKC x3 columns of one plane, 16-byte chunks,
// zero-filled past n3) while the current one is transformed.  Needs n3 a
// multiple of 4 and 16-byte aligned fields (the launcher checks).
template <int N, int TKC, int EPI, typename TO>
__global__ void __launch_bounds__(kThreads)
k_deriv_strided_p(const float *__restrict__ in, TO *out, const float *add, int n3, long long estride,
                  long long pstride, FftPlan p, int ntk, int nitems) {
    extern __shared__ float2 sm[];
    const int n = Fft<N>::size(p);
    float2 *A0 = sm, *A1 = sm + n * TKC, *B = sm + 2 * n * TKC;
    constexpr int CH = TKC / 2;  // 16-byte chunks per row
    auto load = [&](int item, float2 *dst) {
        const int plane = item / ntk, k0 = (item - plane * ntk) * 2 * TKC;
        const float *base = in + (long long)plane * pstride + k0;
        for (int t = threadIdx.x; t < n * CH; t += blockDim.x) {
            const int e = t / CH, ch = t - e * CH;
            const int i3 = k0 + 4 * ch;
            const int bytes = i3 + 4 <= n3 ? 16 : 0;
            cp_async16z(dst + e * TKC + 2 * ch, base + e * estride + (bytes ? 4 * ch : 0), bytes);
        }
        cp_async_commit_all();
    };
    const int i0 = blockIdx.x, stride = gridDim.x;
    if (i0 >= nitems) return;
    load(i0, A0);
    bool cur0 = true;
    const float sc = 1.f / (float)n;
    for (int item = i0; item < nitems; item += stride) {
        float2 *Acur = cur0 ? A0 : A1, *Anext = cur0 ? A1 : A0;
        if (item + stride < nitems) {
            load(item + stride, Anext);
            cp_async_wait_n<1>();
        } else {
            cp_async_wait_n<0>();
        }
        __syncthreads();
        float2 *R = Fft<N>::template run<TKC>(Acur, B, p, TKC, -1.f);
        for (int t = threadIdx.x; t < n * TKC; t += blockDim.x) {
            const int e = t / TKC;
            const float k = wavenumber_d1(e, n) * sc;
            const float2 z = R[t];
            R[t] = make_float2(-k * z.y, k * z.x);
        }
        __syncthreads();
        float2 *S = Fft<N>::template run<TKC>(R, R == Acur ? B : Acur, p, TKC, +1.f);
        const int plane = item / ntk, k0 = (item - plane * ntk) * 2 * TKC;
        const long long base = (long long)plane * pstride;
        for (int t = threadIdx.x; t < n * TKC; t += blockDim.x) {
            const int e = t / TKC, c = t - e * TKC;
            const int i3 = k0 + 2 * c;
            const long long o = base + e * estride + i3;
            const float2 z = S[t];
            if (i3 < n3) {
                float val = z.x;
                if (EPI == EPI_ADD) val += add[o];
                str(out + o, val);
            }
            if (i3 + 1 < n3) {
                float val = z.y;
                if (EPI == EPI_ADD) val += add[o + 1];
                str(out + o + 1, val);
            }
        }
        __syncthreads();
        cur0 = !cur0;
    }
}

// The strided derivative for lengths with an in-place plan (stage_ip): no
// scratch tile, so a block holds only the current and the next tile (three
// blocks per SM at n = 256).  Same transforms and multiplier per line as
// k_deriv_strided_p.
template <int N, int TKC, int EPI, typename TO, int MT, int MINB>
__global__ void __launch_bounds__(MT, MINB)
k_deriv_strided_ip(const float *__restrict__ in, TO *out, const float *add, int n3, long long estride,
                   long long pstride, FftPlan p, int ntk, int nitems) {
    extern __shared__ float2 sm[];
    float2 *cur = sm, *nxt = sm + N * TKC;
    constexpr int CH = TKC / 2;  // 16-byte chunks per row
    const float2 *__restrict__ tw = p.tw;
    auto load = [&](int item, float2 *dst) {
        const int plane = item / ntk, k0 = (item - plane * ntk) * 2 * TKC;
        const float *base = in + (long long)plane * pstride + k0;
        for (int t = threadIdx.x; t < N * CH; t += MT) {
            const int e = t / CH, ch = t - e * CH;
            const int i3 = k0 + 4 * ch;
            const int bytes = i3 + 4 <= n3 ? 16 : 0;
            cp_async16z(dst + e * TKC + 2 * ch, base + e * estride + (bytes ? 4 * ch : 0), bytes);
        }
        cp_async_commit_all();
    };
    const int i0 = blockIdx.x, stride = gridDim.x;
    if (i0 >= nitems) return;
    load(i0, cur);
    const float sc = 1.f / (float)N;
    for (int item = i0; item < nitems; item += stride) {
        if (item + stride < nitems) {
            load(item + stride, nxt);
            cp_async_wait_n<1>();
        } else {
            cp_async_wait_n<0>();
        }
        __syncthreads();
        // forward transform with the multiplier i k / n applied as its last
        // stage stores, then the inverse transform
        const auto deriv = [sc](int e, float2 &z) {
            const float k = wavenumber_d1(e, N) * sc;
            z = make_float2(-k * z.y, k * z.x);
        };
        fft_ip<N, TKC, MT, TKC, 0>(cur, tw, -1.f, deriv);
        fft_ip<N, TKC, MT>(cur, tw, +1.f);
        const int plane = item / ntk, k0 = (item - plane * ntk) * 2 * TKC;
        const long long base = (long long)plane * pstride;
        for (int t = threadIdx.x; t < N * TKC; t += MT) {
            const int e = t / TKC, c = t - e * TKC;
            const int i3 = k0 + 2 * c;
            const long long o = base + e * estride + i3;
            const float2 z = cur[t];
            if (i3 < n3) {
                float val = z.x;
                if (EPI == EPI_ADD) val += add[o];
                str(out + o, val);
            }
            if (i3 + 1 < n3) {
                float val = z.y;
                if (EPI == EPI_ADD) val += add[o + 1];
                str(out + o + 1, val);
            }
        }
        __syncthreads();
        float2 *t = cur;
        cur = nxt;
        nxt = t;
    }
}

// ---- axis derivatives: launchers ------------------------------------------
constexpr int deriv_cols(int n) { return n <= 256 ? 16 : (n <= 512 ? 8 : 4); }

// one instantiation per length and tile; the accumulating form (divergence)
// only for FP32 outputs
template <int N, int L, typename TO>
void deriv_x3_l(const Dims &d, const FftPlan &p, const float *in, TO *out, const float *add, cudaStream_t st) {
    const long long nlines = (long long)d.n1 * d.n2;
    if (d.n3 % 4 == 0 && ((uintptr_t)in & 15) == 0) {
        // the persistent form with the next tile staged by cp.async
        const size_t smem = (fft_in_place(N) ? 1 : 2) * (size_t)d.n3 * (L + 1) * sizeof(float2) +
                            (size_t)2 * L * d.n3 * sizeof(float);
        const int nitems = (int)((nlines + 2 * L - 1) / (2 * L));
        const int grid = persistent_grid(nitems, smem);
        if constexpr (std::is_same<TO, float>::value) {
            if (add) {
                set_smem<k_deriv_x3_p<N, L, EPI_ADD, TO>>(smem);
                k_deriv_x3_p<N, L, EPI_ADD, TO><<<grid, kThreads, smem, st>>>(in, out, add, nlines, p, nitems);
                return;
            }
        }
        set_smem<k_deriv_x3_p<N, L, EPI_STORE, TO>>(smem);
        k_deriv_x3_p<N, L, EPI_STORE, TO><<<grid, kThreads, smem, st>>>(in, out, add, nlines, p, nitems);
        return;
    }
    const size_t smem = 2 * (size_t)d.n3 * (L + 1) * sizeof(float2);
    const unsigned blocks = (unsigned)((nlines + 2 * L - 1) / (2 * L));
    if constexpr (std::is_same<TO, float>::value) {
        if (add) {
            set_smem<k_deriv_x3<N, L, EPI_ADD, TO>>(smem);
            k_deriv_x3<N, L, EPI_ADD, TO><<<blocks, kThreads, smem, st>>>(in, out, add, nlines, p);
            return;
        }
    }
    set_smem<k_deriv_x3<N, L, EPI_STORE, TO>>(smem);
    k_deriv_x3<N, L, EPI_STORE, TO><<<blocks, kThreads, smem, st>>>(in, out, add, nlines, p);
}

template <int N, typename TO>
void deriv_x3_n(const Dims &d, const FftPlan &p, const float *in, TO *out, const float *add, cudaStream_t st) {
    if constexpr (N > 0) {
        deriv_x3_l<N, lines_x3(N)>(d, p, in, out, add, st);
    } else {
        switch (lines_x3(d.n3)) {
            case 16: deriv_x3_l<N, 16>(d, p, in, out, add, st); break;
            case 8: deriv_x3_l<N, 8>(d, p, in, out, add, st); break;
            default: deriv_x3_l<N, 4>(d, p, in, out, add, st); break;
        }
    }
}

template <int N, int TKC, typename TO>
void deriv_strided_t(const Dims &d, const FftPlan &p, int n, const float *in, TO *out, const float *add,
                     long long estride, long long pstride, int nplanes, cudaStream_t st) {
    if constexpr (fft_in_place(N)) {
        if (d.n3 % 4 == 0 && ((uintptr_t)in & 15) == 0) {
            // the in-place double-buffered persistent form
            constexpr int MT = 256;
            constexpr size_t smem = 2 * (size_t)N * TKC * sizeof(float2);
            // three blocks per SM where the registers allow it without spills (n = 128 spills at 85)
            constexpr int MINB = smem <= 72 * 1024 && N >= 256 ? 3 : 2;
            const int ntk = (d.n3 + 2 * TKC - 1) / (2 * TKC), nitems = ntk * nplanes;
            const int grid = persistent_grid(nitems, smem);
            if constexpr (std::is_same<TO, float>::value) {
                if (add) {
                    set_smem<k_deriv_strided_ip<N, TKC, EPI_ADD, TO, MT, MINB>>(smem);
                    k_deriv_strided_ip<N, TKC, EPI_ADD, TO, MT, MINB><<<grid, MT, smem, st>>>(
                        in, out, add, d.n3, estride, pstride, p, ntk, nitems);
                    return;
                }
            }
            set_smem<k_deriv_strided_ip<N, TKC, EPI_STORE, TO, MT, MINB>>(smem);
            k_deriv_strided_ip<N, TKC, EPI_STORE, TO, MT, MINB><<<grid, MT, smem, st>>>(
                in, out, add, d.n3, estride, pstride, p, ntk, nitems);
            return;
        }
    }
    if (d.n3 % 4 == 0 && ((uintptr_t)in & 15) == 0) {
        // the double-buffered persistent form
        const size_t smem = 3 * (size_t)n * TKC * sizeof(float2);
        const int ntk = (d.n3 + 2 * TKC - 1) / (2 * TKC), nitems = ntk * nplanes;
        const int grid = persistent_grid(nitems, smem);
        if constexpr (std::is_same<TO, float>::value) {
            if (add) {
                set_smem<k_deriv_strided_p<N, TKC, EPI_ADD, TO>>(smem);
                k_deriv_strided_p<N, TKC, EPI_ADD, TO><<<grid, kThreads, smem, st>>>(in, out, add, d.n3, estride,
                                                                                   pstride, p, ntk, nitems);
                return;
            }
        }
        set_smem<k_deriv_strided_p<N, TKC, EPI_STORE, TO>>(smem);
        k_deriv_strided_p<N, TKC, EPI_STORE, TO><<<grid, kThreads, smem, st>>>(in, out, add, d.n3, estride, pstride,
                                                                             p, ntk, nitems);
        return;
    }
    const size_t smem = 2 * (size_t)n * TKC * sizeof(float2);
    const dim3 grid((d.n3 + 2 * TKC - 1) / (2 * TKC), nplanes);
    if constexpr (std::is_same<TO, float>::value) {
        if (add) {
            set_smem<k_deriv_strided<N, TKC, EPI_ADD, TO>>(smem);
            k_deriv_strided<N, TKC, EPI_ADD, TO><<<grid, kThreads, smem, st>>>(in, out, add, d.n3, estride, pstride, p);
            return;
        }
    }
    set_smem<k_deriv_strided<N, TKC, EPI_STORE, TO>>(smem);
    k_deriv_strided<N, TKC, EPI_STORE, TO><<<grid, kThreads, smem, st>>>(in, out, add, d.n3, estride, pstride, p);
}

template <int N, typename TO>
void deriv_strided_n(const Dims &d, const FftPlan &p, int n, const float *in, TO *out, const float *add,
                     long long estride, long long pstride, int nplanes, cudaStream_t st) {
    if constexpr (N > 0) {
        deriv_strided_t<N, deriv_cols(N)>(d, p, n, in, out, add, estride, pstride, nplanes, st);
    } else {
        switch (deriv_cols(n)) {
            case 16: deriv_strided_t<N, 16>(d, p, n, in, out, add, estride, pstride, nplanes, st); break;
            case 8: deriv_strided_t<N, 8>(d, p, n, in, out, add, estride, pstride, nplanes, st); break;
            default: deriv_strided_t<N, 4>(d, p, n, in, out, add, estride, pstride, nplanes, st); break;
        }
    }
}

// d/dx_a of in into out (+ add when given); a = 0, 1, 2 for x1, x2, x3
template <typename TO>
void deriv_axis(const Dims &d, const FftPlan *ax, int a, const float *in, TO *out, const float *add,
                cudaStream_t st) {
    const long long plane = (long long)d.n2 * d.n3;
    if (a == 2) {
        switch (d.n3) {
#define CASE_N(NN) case NN: deriv_x3_n<NN>(d, ax[2], in, out, add, st); return;
            CLAIRE_CT_SIZES(CASE_N)
#undef CASE_N
            default: deriv_x3_n<0>(d, ax[2], in, out, add, st);
        }
    } else if (a == 1) {
        switch (d.n2) {
#define CASE_N(NN) case NN: deriv_strided_n<NN>(d, ax[1], d.n2, in, out, add, d.n3, plane, d.n1, st); return;
            CLAIRE_CT_SIZES(CASE_N)
#undef CASE_N
            default: deriv_strided_n<0>(d, ax[1], d.n2, in, out, add, d.n3, plane, d.n1, st);
        }
    } else {
        switch (d.n1) {
#define CASE_N(NN) case NN: deriv_strided_n<NN>(d, ax[0], d.n1, in, out, add, plane, d.n3, d.n2, st); return;
            CLAIRE_CT_SIZES(CASE_N)
#undef CASE_N
            default: deriv_strided_n<0>(d, ax[0], d.n1, in, out, add, plane, d.n3, d.n2, st);
        }
    }
}


}  // namespace

void spectral_grad_1d(const Dims &d, const FftPlan *ax, const float *f, float *g, cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_DERIV, st, 24.0 * d.N, 3);
    for (int a = 0; a < 3; ++a) deriv_axis(d, ax, a, f, g + (size_t)a * d.N, nullptr, st);
}

void spectral_grad_1d(const Dims &d, const FftPlan *ax, const float *f, __half *g, cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_DERIV, st, 18.0 * d.N, 3);
    for (int a = 0; a < 3; ++a) deriv_axis(d, ax, a, f, g + (size_t)a * d.N, nullptr, st);
}

void spectral_div_1d(const Dims &d, const FftPlan *ax, const float *v, float *out, cudaStream_t st, Profiler *prof) {
    ProfScope ps(prof, CLAIRE_K_DERIV, st, 32.0 * d.N, 3);
    deriv_axis(d, ax, 2, v + 2 * (size_t)d.N, out, (const float *)nullptr, st);
    deriv_axis(d, ax, 1, v + (size_t)d.N, out, out, st);
    deriv_axis(d, ax, 0, v, out, out, st);
}

}  // namespace claire
