// deriv.cu -- eighth-order central finite differences for first derivatives
// (paper Section 4.2), the paper's GPU alternative to spectral differentiation:
//   df/dx_d (x) ~ (1/h_d) sum_{j=1..4} c_j (f(x + j e_d) - f(x - j e_d)),
//   c = (4/5, -1/5, 4/105, -1/280), periodic.
// One thread per voxel, a block covering 32 consecutive x3 points of 8 x2
// rows; the 24 neighbours come through L1 (x3 neighbours are in the same or
// the adjacent cache line, x2 and x1 neighbours are reused by nearby blocks).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "claire_internal.cuh"

namespace claire {

namespace {

constexpr int DX = 32, DY = 8;

__device__ __forceinline__ int wrapn(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// outputs are FP32, or FP16 in the FP16-storage form (FP32 arithmetic)
__device__ __forceinline__ float ldd(const float *p) { return __ldg(p); }
__device__ __forceinline__ void std_(float *p, float v) { *p = v; }
__device__ __forceinline__ void std_(__half *p, float v) { *p = __float2half_rn(v); }

// derivative along axis d (stride s, length n, position i) of f at base offset o
template <typename T>
__device__ __forceinline__ float fd8(const T *__restrict__ f, long long o, int i, int n,
                                     long long s, float ih) {
    const float c1 = 4.f / 5.f, c2 = -1.f / 5.f, c3 = 4.f / 105.f, c4 = -1.f / 280.f;
    const long long b = o - (long long)i * s;  // offset of index 0 on this line
    auto at = [&](int k) { return ldd(f + b + (long long)wrapn(i + k, n) * s); };
    float r = c4 * (at(4) - at(-4));
    r = fmaf(c3, at(3) - at(-3), r);
    r = fmaf(c2, at(2) - at(-2), r);
    r = fmaf(c1, at(1) - at(-1), r);
    return r * ih;
}

template <typename TO>
__global__ void __launch_bounds__(DX * DY) k_grad_fd8(const float *__restrict__ f, TO *__restrict__ g,
                                                      Dims d, float ih1, float ih2, float ih3) {
    const int i3 = blockIdx.x * DX + threadIdx.x, i2 = blockIdx.y * DY + threadIdx.y, i1 = blockIdx.z;
    if (i3 >= d.n3 || i2 >= d.n2) return;
    const long long s1 = (long long)d.n2 * d.n3, s2 = d.n3;
    const long long o = i1 * s1 + i2 * s2 + i3;
    std_(g + o, fd8(f, o, i1, d.n1, s1, ih1));
    std_(g + d.N + o, fd8(f, o, i2, d.n2, s2, ih2));
    std_(g + 2 * d.N + o, fd8(f, o, i3, d.n3, 1, ih3));
}

__global__ void __launch_bounds__(DX * DY) k_div_fd8(const float *__restrict__ v, float *__restrict__ out,
                                                     Dims d, float ih1, float ih2, float ih3) {
    const int i3 = blockIdx.x * DX + threadIdx.x, i2 = blockIdx.y * DY + threadIdx.y, i1 = blockIdx.z;
    if (i3 >= d.n3 || i2 >= d.n2) return;
    const long long s1 = (long long)d.n2 * d.n3, s2 = d.n3;
    const long long o = i1 * s1 + i2 * s2 + i3;
    out[o] = fd8(v, o, i1, d.n1, s1, ih1) + fd8(v + d.N, o, i2, d.n2, s2, ih2) +
             fd8(v + 2 * d.N, o, i3, d.n3, 1, ih3);
}

inline dim3 grid_d(const Dims &d) { return dim3((d.n3 + DX - 1) / DX, (d.n2 + DY - 1) / DY, d.n1); }

}  // namespace

void launch_grad_fd8(const Dims &d, const float *f, float *g, cudaStream_t st, Profiler *prof) {
    const double tp = 6.283185307179586476925286766559;
    ProfScope ps(prof, CLAIRE_K_FD, st, 16.0 * d.N);
    k_grad_fd8<<<grid_d(d), dim3(DX, DY), 0, st>>>(f, g, d, (float)(d.n1 / tp), (float)(d.n2 / tp),
                                                   (float)(d.n3 / tp));
}

void launch_grad_fd8(const Dims &d, const float *f, __half *g, cudaStream_t st, Profiler *prof) {
    const double tp = 6.283185307179586476925286766559;
    ProfScope ps(prof, CLAIRE_K_FD, st, 10.0 * d.N);
    k_grad_fd8<<<grid_d(d), dim3(DX, DY), 0, st>>>(f, g, d, (float)(d.n1 / tp), (float)(d.n2 / tp),
                                                   (float)(d.n3 / tp));
}

void launch_div_fd8(const Dims &d, const float *v, float *out, cudaStream_t st, Profiler *prof) {
    const double tp = 6.283185307179586476925286766559;
    ProfScope ps(prof, CLAIRE_K_FD, st, 16.0 * d.N);
    k_div_fd8<<<grid_d(d), dim3(DX, DY), 0, st>>>(v, out, d, (float)(d.n1 / tp), (float)(d.n2 / tp),
                                                  (float)(d.n3 / tp));
}

}  // namespace claire
