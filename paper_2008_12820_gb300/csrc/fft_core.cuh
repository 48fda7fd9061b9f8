// fft_core.cuh -- the shared-memory Stockham FFT building blocks of the
// pencil transforms (fft.cu) and the axis derivatives (fft_axis.cu): in-register
// DFTs of radix 2, 3, 4, 5, 8, 16, the Stockham stages (out of place with a
// scratch tile, and in place for power-of-two lengths from 128), compile-time
// plans for the common lengths and a runtime plan for the others, wavenumbers,
// and the launch helpers.  Internal linkage: each translation unit instantiates what
// it uses.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "claire_internal.cuh"

namespace claire {
namespace {

// real fields are FP32, or FP16 in the FP16-storage form (FP32 arithmetic)
__device__ __forceinline__ float ldr(const float *p) { return *p; }
__device__ __forceinline__ void str(float *p, float v) { *p = v; }
__device__ __forceinline__ void str(__half *p, float v) { *p = __float2half_rn(v); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// multiply by s*i (s = +-1)
__device__ __forceinline__ float2 mul_si(float2 a, float s) { return make_float2(-s * a.y, s * a.x); }

// in-register DFT of size R: X_q = sum_r a_r exp(s 2 pi i r q / R)
template <int R> __device__ __forceinline__ void dft(float2 *a, float s);

template <> __device__ __forceinline__ void dft<2>(float2 *a, float) {
    float2 t = a[1];
    a[1] = csub(a[0], t);
    a[0] = cadd(a[0], t);
}

template <> __device__ __forceinline__ void dft<3>(float2 *a, float s) {
    const float c = 0.86602540378443864676f;  // sqrt(3)/2
    float2 t1 = cadd(a[1], a[2]);
    float2 t2 = csub(a[1], a[2]);
    float2 m = make_float2(a[0].x - 0.5f * t1.x, a[0].y - 0.5f * t1.y);
    float2 r = mul_si(make_float2(c * t2.x, c * t2.y), s);
    a[0] = cadd(a[0], t1);
    a[1] = cadd(m, r);
    a[2] = csub(m, r);
}

template <> __device__ __forceinline__ void dft<4>(float2 *a, float s) {
    float2 t0 = cadd(a[0], a[2]);
    float2 t1 = csub(a[0], a[2]);
    float2 t2 = cadd(a[1], a[3]);
    float2 t3 = mul_si(csub(a[1], a[3]), s);
    a[0] = cadd(t0, t2);
    a[2] = csub(t0, t2);
    a[1] = cadd(t1, t3);
    a[3] = csub(t1, t3);
}

template <> __device__ __forceinline__ void dft<5>(float2 *a, float s) {
    const float c1 = 0.30901699437494742410f;   // cos(2 pi / 5)
    const float c2 = -0.80901699437494742410f;  // cos(4 pi / 5)
    const float s1 = 0.95105651629515357212f;   // sin(2 pi / 5)
    const float s2 = 0.58778525229247312917f;   // sin(4 pi / 5)
    float2 t1 = cadd(a[1], a[4]), t2 = cadd(a[2], a[3]);
    float2 t3 = csub(a[1], a[4]), t4 = csub(a[2], a[3]);
    float2 b1 = make_float2(a[0].x + c1 * t1.x + c2 * t2.x, a[0].y + c1 * t1.y + c2 * t2.y);
    float2 b2 = make_float2(a[0].x + c2 * t1.x + c1 * t2.x, a[0].y + c2 * t1.y + c1 * t2.y);
    float2 e1 = mul_si(make_float2(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y), s);
    float2 e2 = mul_si(make_float2(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y), s);
    a[0] = make_float2(a[0].x + t1.x + t2.x, a[0].y + t1.y + t2.y);
    a[1] = cadd(b1, e1);
    a[4] = csub(b1, e1);
    a[2] = cadd(b2, e2);
    a[3] = csub(b2, e2);
}

template <> __device__ __forceinline__ void dft<8>(float2 *a, float s) {
    const float h = 0.70710678118654752440f;  // cos(pi/4)
    float2 e[4] = {a[0], a[2], a[4], a[6]};
    float2 o[4] = {a[1], a[3], a[5], a[7]};
    dft<4>(e, s);
    dft<4>(o, s);
    // o_q *= exp(s 2 pi i q / 8)
    o[1] = cmul(o[1], make_float2(h, s * h));
    o[2] = mul_si(o[2], s);
    o[3] = cmul(o[3], make_float2(-h, s * h));
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        a[q] = cadd(e[q], o[q]);
        a[q + 4] = csub(e[q], o[q]);
    }
}

// 16 = 4 x 4: DFT-4 over r2 for each r1, twiddle exp(s 2 pi i r1 q1 / 16),
// DFT-4 over r1 for each q1; output index q1 + 4 q2
template <> __device__ __forceinline__ void dft<16>(float2 *a, float s) {
    const float c1 = 0.92387953251128675613f;  // cos(pi/8)
    const float s1 = 0.38268343236508977173f;  // sin(pi/8)
    const float h = 0.70710678118654752440f;
    float2 y[4][4];
#pragma unroll
    for (int r1 = 0; r1 < 4; ++r1) {
        float2 t[4] = {a[r1], a[r1 + 4], a[r1 + 8], a[r1 + 12]};
        dft<4>(t, s);
#pragma unroll
        for (int q1 = 0; q1 < 4; ++q1) y[r1][q1] = t[q1];
    }
    y[1][1] = cmul(y[1][1], make_float2(c1, s * s1));   // e = 1
    y[1][2] = cmul(y[1][2], make_float2(h, s * h));     // e = 2
    y[1][3] = cmul(y[1][3], make_float2(s1, s * c1));   // e = 3
    y[2][1] = cmul(y[2][1], make_float2(h, s * h));     // e = 2
    y[2][2] = mul_si(y[2][2], s);                       // e = 4
    y[2][3] = cmul(y[2][3], make_float2(-h, s * h));    // e = 6
    y[3][1] = cmul(y[3][1], make_float2(s1, s * c1));   // e = 3
    y[3][2] = cmul(y[3][2], make_float2(-h, s * h));    // e = 6
    y[3][3] = cmul(y[3][3], make_float2(-c1, -s * s1)); // e = 9
#pragma unroll
    for (int q1 = 0; q1 < 4; ++q1) {
        float2 t[4] = {y[0][q1], y[1][q1], y[2][q1], y[3][q1]};
        dft<4>(t, s);
#pragma unroll
        for (int q2 = 0; q2 < 4; ++q2) a[q1 + 4 * q2] = t[q2];
    }
}

// One Stockham stage of radix R over L lines stored as buf[e * ls + l]
// (e = element index, l = line).  Ns = product of the earlier radices.
template <int R, int L>
__device__ __forceinline__ void stage(const float2 *__restrict__ A, float2 *__restrict__ B,
                                      int n, int Ns, int ls, const float2 *__restrict__ tw,
                                      float s) {
    const int nb = n / R;
    const int work = nb * L;
    const int tstride = n / (Ns * R);
    for (int t = threadIdx.x; t < work; t += blockDim.x) {
        const int l = t % L;
        const int j = t / L;
        const int k = j % Ns;
        float2 a[R];
#pragma unroll
        for (int r = 0; r < R; ++r) a[r] = A[(j + r * nb) * ls + l];
        if (k != 0) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = __ldg(tw + r * k * tstride);
                w.y *= -s;  // table holds exp(-2 pi i t/n); s = +1 conjugates
                a[r] = cmul(a[r], w);
            }
        }
        dft<R>(a, s);
        const int base = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) B[(base + r * Ns) * ls + l] = a[r];
    }
}

// Full FFT of L lines of length p.n, data in A, B as scratch.  s = -1
// forward, +1 inverse (unnormalized).  Returns the buffer holding the result.
// Leaves a __syncthreads() after every stage.
template <int L>
__device__ float2 *fft_lines(float2 *A, float2 *B, const FftPlan &p, int ls, float s) {
    int Ns = 1;
    for (int st = 0; st < p.nst; ++st) {
        const int R = p.rad[st];
        switch (R) {
            case 2: stage<2, L>(A, B, p.n, Ns, ls, p.tw, s); break;
            case 3: stage<3, L>(A, B, p.n, Ns, ls, p.tw, s); break;
            case 4: stage<4, L>(A, B, p.n, Ns, ls, p.tw, s); break;
            default: stage<5, L>(A, B, p.n, Ns, ls, p.tw, s); break;
        }
        __syncthreads();
        float2 *t = A;
        A = B;
        B = t;
        Ns *= R;
    }
    return A;
}

// ---------------------------------------------------------------------------
// Compile-time plans for the common grid sizes: radix 16 while it divides the
// power-of-two part, then one 8, 4 or 2, then 3s, then 5s.  With the length,
// radices and strides known, every index division folds into shifts or
// multiplications and the loops unroll; radix 8 and 16 keep more of the
// transform in registers (fewer shared-memory passes and barriers).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int pow2_part(int n) {
    int p = 1;
    while (n % 2 == 0) { n /= 2; p *= 2; }
    return p;
}
__host__ __device__ constexpr int radix_at(int n, int s) {
    int p2 = pow2_part(n), rest = n / p2, st = 0;
    while (p2 >= 16) { if (st == s) return 16; p2 /= 16; ++st; }
    if (p2 > 1) { if (st == s) return p2; ++st; }
    while (rest % 3 == 0) { if (st == s) return 3; rest /= 3; ++st; }
    while (rest % 5 == 0) { if (st == s) return 5; rest /= 5; ++st; }
    return 0;
}
__host__ __device__ constexpr int num_stages(int n) {
    int s = 0;
    while (radix_at(n, s) != 0) ++s;
    return s;
}
__host__ __device__ constexpr int ns_before(int n, int s) {
    int p = 1;
    for (int i = 0; i < s; ++i) p *= radix_at(n, i);
    return p;
}

template <int N, int R, int NS, int L>
__device__ __forceinline__ void stage_ct(const float2 *__restrict__ A, float2 *__restrict__ B,
                                         int ls, const float2 *__restrict__ tw, float s) {
    constexpr int NB = N / R, WORK = NB * L, TSTRIDE = N / (NS * R);
#pragma unroll 2
    for (int t = threadIdx.x; t < WORK; t += kThreads) {
        const int l = t % L;
        const int j = t / L;
        const int k = j % NS;
        float2 a[R];
#pragma unroll
        for (int r = 0; r < R; ++r) a[r] = A[(j + r * NB) * ls + l];
        if (NS > 1 && k != 0) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = __ldg(tw + r * k * TSTRIDE);
                w.y *= -s;
                a[r] = cmul(a[r], w);
            }
        }
        dft<R>(a, s);
        const int base = (j / NS) * NS * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) B[(base + r * NS) * ls + l] = a[r];
    }
}

template <int N, int L, int S = 0>
__device__ __forceinline__ float2 *fft_ct(float2 *A, float2 *B, const float2 *__restrict__ tw,
                                          int ls, float s) {
    if constexpr (S == num_stages(N)) {
        return A;
    } else {
        stage_ct<N, radix_at(N, S), ns_before(N, S), L>(A, B, ls, tw, s);
        __syncthreads();
        return fft_ct<N, L, S + 1>(B, A, tw, ls, s);
    }
}

// In-place form of the compile-time plan for NT threads: each thread reads all
// of its butterflies of a stage into registers (IT of them), the block waits,
// and the results go back into the same buffer.  No scratch buffer, so a
// block can hold more lines in the same shared memory, and with WORK a
// multiple of NT every thread has work in every stage.  Same butterflies,
// twiddles and order of operations per line as stage_ct.
// no pointwise step after the last stage
struct NoPost {
    __device__ __forceinline__ void operator()(int, float2 &) const {}
};

template <int N, int R, int NS, int L, int NT, int LS = L, class Post = NoPost>
__device__ __forceinline__ void stage_ip(float2 *__restrict__ A, const float2 *__restrict__ tw, float s,
                                         const Post &post = Post()) {
    constexpr int NB = N / R, WORK = NB * L, TSTRIDE = N / (NS * R), IT = (WORK + NT - 1) / NT;
    float2 a[IT][R];
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        const int t = threadIdx.x + i * NT;
        if (WORK % NT == 0 || t < WORK) {
            const int l = t % L;
            const int j = t / L;
            const int k = j % NS;
#pragma unroll
            for (int r = 0; r < R; ++r) a[i][r] = A[(j + r * NB) * LS + l];
            if (NS > 1 && k != 0) {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    float2 w = __ldg(tw + r * k * TSTRIDE);
                    w.y *= -s;
                    a[i][r] = cmul(a[i][r], w);
                }
            }
            dft<R>(a[i], s);
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        const int t = threadIdx.x + i * NT;
        if (WORK % NT == 0 || t < WORK) {
            const int l = t % L;
            const int j = t / L;
            const int k = j % NS;
            const int base = (j / NS) * NS * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                post(base + r * NS, a[i][r]);
                A[(base + r * NS) * LS + l] = a[i][r];
            }
        }
    }
    __syncthreads();
}

// FFT of L lines of length N stored as A[e * LS + l] (LS >= L; an odd LS
// keeps the transposing loads of the x3 passes free of bank conflicts), in
// place, NT threads; ends behind a barrier.  post(e, v) is applied to every
// output element (e = its index along the line) before the last stage
// stores it: a pointwise multiplier without another pass over the tile.
template <int N, int L, int NT, int LS = L, int S = 0, class Post = NoPost>
__device__ __forceinline__ void fft_ip(float2 *A, const float2 *__restrict__ tw, float s,
                                       const Post &post = Post()) {
    if constexpr (S + 1 == num_stages(N)) {
        stage_ip<N, radix_at(N, S), ns_before(N, S), L, NT, LS, Post>(A, tw, s, post);
    } else if constexpr (S < num_stages(N)) {
        stage_ip<N, radix_at(N, S), ns_before(N, S), L, NT, LS>(A, tw, s);
        fft_ip<N, L, NT, LS, S + 1, Post>(A, tw, s, post);
    }
}

// The lengths whose passes use the in-place plan: powers of two from 128 on
// (radix-16 stages with one or two butterflies a thread, no register spills);
// the other lengths keep the out-of-place stages with a scratch tile.
__host__ __device__ constexpr bool fft_in_place(int n) { return n >= 128 && (n & (n - 1)) == 0; }

// N > 0: compile-time plan of that length; N == 0: the runtime plan p
template <int N>
struct Fft {
    __device__ __forceinline__ static int size(const FftPlan &p) { return N > 0 ? N : p.n; }
    template <int L>
    __device__ __forceinline__ static float2 *run(float2 *A, float2 *B, const FftPlan &p, int ls,
                                                  float s) {
        if constexpr (N > 0) return fft_ct<N, L>(A, B, p.tw, ls, s);
        else return fft_lines<L>(A, B, p, ls, s);
    }
};

__device__ __forceinline__ float wavenumber(int i, int n) { return (2 * i < n) ? (float)i : (float)(i - n); }
__device__ __forceinline__ float wavenumber_d1(int i, int n) {
    return ((n & 1) == 0 && 2 * i == n) ? 0.f : wavenumber(i, n);
}

// ------------------------------------------------------- launch helpers --

// dynamic shared-memory limit of a transform kernel: one SmemAttr per kernel
// instantiation (set per device, failures reported with a clear message)
template <auto K>
void set_smem(size_t bytes) {
    static SmemAttr a;
    a.ensure(K, (int)bytes, "pencil FFT pass");
}

// 16-byte cp.async of `bytes` (0, 8 or 16) valid bytes, the rest zero-filled
__device__ __forceinline__ void cp_async16z(void *smem, const void *gmem, int bytes) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit_all() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int NPEND>
__device__ __forceinline__ void cp_async_wait_n() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(NPEND) : "memory");
}

// lines per block of the x3 passes and column tile of the strided passes,
// chosen so that a block's shared memory stays near or below ~112 KB
constexpr int lines_x3(int n) { return n <= 256 ? 16 : (n <= 512 ? 8 : 4); }
constexpr int tile_cols(int n, int nbuf) {
    // nbuf data buffers + one scratch of n*TK float2
    return (size_t)(nbuf + 1) * n * 16 * sizeof(float2) <= 112 * 1024 ? 16
         : (size_t)(nbuf + 1) * n * 8 * sizeof(float2) <= 112 * 1024 ? 8 : 4;
}

// the axis lengths with a compile-time plan; other valid lengths use the
// runtime plan (N = 0)
#define CLAIRE_CT_SIZES(X) X(32) X(64) X(96) X(128) X(160) X(192) X(256) X(384) X(512) X(768)

}  // namespace
}  // namespace claire
