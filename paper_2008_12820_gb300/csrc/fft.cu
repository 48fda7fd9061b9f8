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
#include <cuda_runtime.h>

#include "claire_internal.cuh"

namespace claire {

namespace {

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

// ---------------------------------------------------------------- pass 1 ---
// x3 forward real -> half spectrum.  Block: L complex lines = 2L real lines.
template <int L>
__global__ void __launch_bounds__(kThreads)
k_r2c_x3(const float *__restrict__ in, float2 *__restrict__ out, long long nlines, FftPlan p,
         int h3, int p3) {
    extern __shared__ float2 sm[];
    const int n = p.n, ls = L + 1;
    float2 *A = sm, *B = sm + n * ls;
    const long long line0 = (long long)blockIdx.x * 2 * L;
    float *Af = reinterpret_cast<float *>(A);
    for (int t = threadIdx.x; t < 2 * L * n; t += blockDim.x) {
        const int rl = t / n, e = t - rl * n;
        const long long line = line0 + rl;
        const float val = line < nlines ? in[line * n + e] : 0.f;
        Af[(e * ls + (rl >> 1)) * 2 + (rl & 1)] = val;
    }
    __syncthreads();
    float2 *Rz = fft_lines<L>(A, B, p, ls, -1.f);
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

// ---------------------------------------------------------------- pass 2 ---
// x2 complex transform in place.  Block: (k3 tile of TK, one (c, i1) plane).
template <int TK>
__global__ void __launch_bounds__(kThreads)
k_c2c_x2(float2 *__restrict__ data, FftPlan p, int h3, int p3, float s) {
    extern __shared__ float2 sm[];
    const int n = p.n;
    float2 *A = sm, *B = sm + n * TK;
    float2 *base = data + (long long)blockIdx.y * n * p3;
    const int k0 = blockIdx.x * TK;
    for (int t = threadIdx.x; t < n * TK; t += blockDim.x) {
        const int e = t / TK, l = t - e * TK;
        A[e * TK + l] = (k0 + l < h3) ? base[(long long)e * p3 + k0 + l] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2 *R = fft_lines<TK>(A, B, p, TK, s);
    for (int t = threadIdx.x; t < n * TK; t += blockDim.x) {
        const int e = t / TK, l = t - e * TK;
        if (k0 + l < h3) base[(long long)e * p3 + k0 + l] = R[e * TK + l];
    }
}

__device__ __forceinline__ float wavenumber(int i, int n) { return (2 * i < n) ? (float)i : (float)(i - n); }
__device__ __forceinline__ float wavenumber_d1(int i, int n) {
    return ((n & 1) == 0 && 2 * i == n) ? 0.f : wavenumber(i, n);
}

// ---------------------------------------------------------------- pass 3 ---
// x1 forward, multiplier, x1 inverse, in place.  Block: (k3 tile, k2 index).
// Buffers: NB = max(nin, nout) component tiles of n1*TK plus one scratch.
template <int TK, int OP>
__global__ void __launch_bounds__(kThreads)
k_mul_x1(float2 *__restrict__ data, FftPlan p1, int n2, int n3, int h3, int p3,
         long long cstride, SpecParams sp) {
    constexpr int NIN = (OP == OP_GRAD) ? 1 : 3;
    constexpr int NOUT = (OP == OP_DIV) ? 1 : 3;
    constexpr int NB = NIN > NOUT ? NIN : NOUT;
    extern __shared__ float2 sm[];
    const int n1 = p1.n;
    const int tile = n1 * TK;
    float2 *buf[NB];
    float2 *scratch = sm + NB * tile;
#pragma unroll
    for (int c = 0; c < NB; ++c) buf[c] = sm + c * tile;
    const int i2 = blockIdx.y;
    const int k0 = blockIdx.x * TK;
    const long long rowstride = (long long)n2 * p3;  // between consecutive i1
    float2 *base = data + (long long)i2 * p3 + k0;
    for (int c = 0; c < NIN; ++c) {
        for (int t = threadIdx.x; t < tile; t += blockDim.x) {
            const int e = t / TK, l = t - e * TK;
            buf[c][e * TK + l] = (k0 + l < h3) ? base[c * cstride + e * rowstride + l]
                                               : make_float2(0.f, 0.f);
        }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NIN; ++c) {
        float2 *r = fft_lines<TK>(buf[c], scratch, p1, TK, -1.f);
        if (r != buf[c]) { scratch = buf[c]; buf[c] = r; }
    }
    // multiplier at (k1, k2, k3)
    const float k2 = wavenumber(i2, n2), k2d = wavenumber_d1(i2, n2);
    for (int t = threadIdx.x; t < tile; t += blockDim.x) {
        const int e = t / TK, l = t - e * TK;
        const int i3 = k0 + l;
        const float k1 = wavenumber(e, n1), k1d = wavenumber_d1(e, n1);
        const float k3 = (float)i3, k3d = ((n3 & 1) == 0 && 2 * i3 == n3) ? 0.f : k3;
        const int id = e * TK + l;
        if (OP == OP_GRAD) {
            const float2 f = buf[0][id];
            // i k_d f * scale
            buf[0][id] = make_float2(-k1d * f.y * sp.scale, k1d * f.x * sp.scale);
            buf[1][id] = make_float2(-k2d * f.y * sp.scale, k2d * f.x * sp.scale);
            buf[2][id] = make_float2(-k3d * f.y * sp.scale, k3d * f.x * sp.scale);
        } else if (OP == OP_DIV) {
            const float2 a = buf[0][id], b = buf[1][id], c = buf[2][id];
            const float re = k1d * a.x + k2d * b.x + k3d * c.x;
            const float im = k1d * a.y + k2d * b.y + k3d * c.y;
            buf[0][id] = make_float2(-im * sp.scale, re * sp.scale);
        } else {
            const float2 a = buf[0][id], b = buf[1][id], c = buf[2][id];
            const float kk = k1 * k1 + k2 * k2 + k3 * k3;
            const float kd2 = k1d * k1d + k2d * k2d + k3d * k3d;
            // khat . v
            const float2 kv = make_float2(k1d * a.x + k2d * b.x + k3d * c.x,
                                          k1d * a.y + k2d * b.y + k3d * c.y);
            float diag, coup;
            if (OP == OP_A) {
                // (beta |k|^2 I + gamma khat khat^T) v
                diag = sp.beta * kk;
                coup = sp.gamma;
            } else {
                // (beta |k|^2)^-1 (I - gamma khat khat^T / (beta |k|^2 + gamma |khat|^2)) v,
                // identity at k = 0 (Sherman-Morrison)
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
            buf[0][id] = make_float2((diag * a.x + coup * k1d * kv.x) * s, (diag * a.y + coup * k1d * kv.y) * s);
            buf[1][id] = make_float2((diag * b.x + coup * k2d * kv.x) * s, (diag * b.y + coup * k2d * kv.y) * s);
            buf[2][id] = make_float2((diag * c.x + coup * k3d * kv.x) * s, (diag * c.y + coup * k3d * kv.y) * s);
        }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NOUT; ++c) {
        float2 *r = fft_lines<TK>(buf[c], scratch, p1, TK, +1.f);
        if (r != buf[c]) { scratch = buf[c]; buf[c] = r; }
    }
    for (int c = 0; c < NOUT; ++c) {
        for (int t = threadIdx.x; t < tile; t += blockDim.x) {
            const int e = t / TK, l = t - e * TK;
            if (k0 + l < h3) base[c * cstride + e * rowstride + l] = buf[c][e * TK + l];
        }
    }
}

// ---------------------------------------------------------------- pass 5 ---
// x3 inverse half spectrum -> real, two real lines per complex transform.
template <int L, int EPI>
__global__ void __launch_bounds__(kThreads)
k_c2r_x3(const float2 *__restrict__ in, float *__restrict__ out, const float *__restrict__ add,
         long long nlines, FftPlan p, int h3, int p3) {
    extern __shared__ float2 sm[];
    const int n = p.n, ls = L + 1;
    float2 *A = sm, *B = sm + n * ls;
    const long long line0 = (long long)blockIdx.x * 2 * L;
    const bool even = (n & 1) == 0;
    for (int t = threadIdx.x; t < L * n; t += blockDim.x) {
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
    float2 *R = fft_lines<L>(A, B, p, ls, +1.f);
    const float *Rf = reinterpret_cast<const float *>(R);
    for (int t = threadIdx.x; t < 2 * L * n; t += blockDim.x) {
        const int rl = t / n, e = t - rl * n;
        const long long line = line0 + rl;
        if (line < nlines) {
            float val = Rf[(e * ls + (rl >> 1)) * 2 + (rl & 1)];
            if (EPI == EPI_ADD) val += add[line * n + e];
            out[line * n + e] = val;
        }
    }
}

// -------------------------------------------------------------- launchers --

template <typename K>
void set_smem(K kernel, size_t bytes) {
    if (bytes > 48 * 1024)
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// lines per block of the x3 passes and column tile of the strided passes,
// chosen so that a block's shared memory stays near or below ~110 KB
int lines_x3(int n) { return n <= 256 ? 16 : (n <= 512 ? 8 : 4); }
int tile_x1(int n, int nbuf) {
    // nbuf buffers + scratch of n*TK float2
    for (int tk = 16; tk >= 4; tk /= 2)
        if ((size_t)(nbuf + 1) * n * tk * sizeof(float2) <= 112 * 1024) return tk;
    return 4;
}

void r2c_x3(const Dims &d, const FftPlan &p, const float *in, float2 *out, int ncomp,
            cudaStream_t st) {
    const long long nlines = (long long)ncomp * d.n1 * d.n2;
    const int L = lines_x3(d.n3);
    const size_t smem = 2 * (size_t)d.n3 * (L + 1) * sizeof(float2);
    const long long blocks = (nlines + 2 * L - 1) / (2 * L);
#define R2C_CASE(LL)                                                                     \
    case LL:                                                                             \
        set_smem(k_r2c_x3<LL>, smem);                                                    \
        k_r2c_x3<LL><<<(unsigned)blocks, kThreads, smem, st>>>(in, out, nlines, p, d.h3, d.p3); \
        break;
    switch (L) { R2C_CASE(16) R2C_CASE(8) R2C_CASE(4) }
#undef R2C_CASE
}

void c2c_x2(const Dims &d, const FftPlan &p, float2 *data, int ncomp, float s, cudaStream_t st) {
    const int TK = tile_x1(d.n2, 1);
    const size_t smem = 2 * (size_t)d.n2 * TK * sizeof(float2);
    dim3 grid((d.h3 + TK - 1) / TK, ncomp * d.n1);
#define C2C_CASE(T)                                                            \
    case T:                                                                    \
        set_smem(k_c2c_x2<T>, smem);                                           \
        k_c2c_x2<T><<<grid, kThreads, smem, st>>>(data, p, d.h3, d.p3, s);     \
        break;
    switch (TK) { C2C_CASE(16) C2C_CASE(8) C2C_CASE(4) }
#undef C2C_CASE
}

template <int OP>
void mul_x1_op(const Dims &d, const FftPlan &p, float2 *data, const SpecParams &sp,
               cudaStream_t st) {
    constexpr int NIN = (OP == OP_GRAD) ? 1 : 3;
    constexpr int NOUT = (OP == OP_DIV) ? 1 : 3;
    constexpr int NB = NIN > NOUT ? NIN : NOUT;
    const int TK = tile_x1(d.n1, NB);
    const size_t smem = (size_t)(NB + 1) * d.n1 * TK * sizeof(float2);
    const long long cstride = (long long)d.n1 * d.n2 * d.p3;
    dim3 grid((d.h3 + TK - 1) / TK, d.n2);
#define MUL_CASE(T)                                                                          \
    case T:                                                                                  \
        set_smem(k_mul_x1<T, OP>, smem);                                                     \
        k_mul_x1<T, OP><<<grid, kThreads, smem, st>>>(data, p, d.n2, d.n3, d.h3, d.p3,       \
                                                       cstride, sp);                          \
        break;
    switch (TK) { MUL_CASE(16) MUL_CASE(8) MUL_CASE(4) }
#undef MUL_CASE
}

void c2r_x3(const Dims &d, const FftPlan &p, const float2 *in, float *out, const float *add,
            int ncomp, cudaStream_t st) {
    const long long nlines = (long long)ncomp * d.n1 * d.n2;
    const int L = lines_x3(d.n3);
    const size_t smem = 2 * (size_t)d.n3 * (L + 1) * sizeof(float2);
    const long long blocks = (nlines + 2 * L - 1) / (2 * L);
#define C2R_CASE(LL, E)                                                                    \
    set_smem(k_c2r_x3<LL, E>, smem);                                                       \
    k_c2r_x3<LL, E><<<(unsigned)blocks, kThreads, smem, st>>>(in, out, add, nlines, p, d.h3, d.p3);
    if (add) {
        switch (L) {
            case 16: C2R_CASE(16, EPI_ADD) break;
            case 8: C2R_CASE(8, EPI_ADD) break;
            default: C2R_CASE(4, EPI_ADD) break;
        }
    } else {
        switch (L) {
            case 16: C2R_CASE(16, EPI_STORE) break;
            case 8: C2R_CASE(8, EPI_STORE) break;
            default: C2R_CASE(4, EPI_STORE) break;
        }
    }
#undef C2R_CASE
}

}  // namespace

void spectral_apply(const Dims &d, const FftPlan *ax, SpecOp op, const SpecParams &sp,
                    const float *in, float *out, const float *add, float2 *spec, cudaStream_t st,
                    Profiler *prof) {
    const int nin = (op == OP_GRAD) ? 1 : 3;
    const int nout = (op == OP_DIV) ? 1 : 3;
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
            case OP_GRAD: mul_x1_op<OP_GRAD>(d, ax[0], spec, sp, st); break;
            case OP_DIV: mul_x1_op<OP_DIV>(d, ax[0], spec, sp, st); break;
            case OP_A: mul_x1_op<OP_A>(d, ax[0], spec, sp, st); break;
            default: mul_x1_op<OP_AINV>(d, ax[0], spec, sp, st); break;
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
