// reduce.cuh -- compensated FP32 accumulation and FP64 block sums, shared by
// the vector kernels and the semi-Lagrangian steps that fold a dot product
// into their epilogue.
//
// A thread accumulates its elements with error-free transformations in FP32
// (the compensated dot product of Ogita, Rump and Oishi, "Accurate sum and
// dot product", SIAM J. Sci. Comput. 2005: TwoProduct by fma, TwoSum by
// Knuth), as accurate as summing in twice the working precision; the pair
// (sum, compensation) is widened to FP64 once and a block reduces in FP64 by
// warp shuffles.  Internal linkage: every translation unit gets its own copy.
#pragma once

#include <cuda_runtime.h>

namespace claire {
namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// sum of v over a block of NT threads (lin: the thread's linear index);
// valid in the thread with lin == 0
template <int NT>
__device__ __forceinline__ double block_sum_n(double v, int lin) {
    static_assert(NT % 32 == 0 && NT <= 1024, "whole warps");
    __shared__ double ws[NT / 32];
    v = warp_sum(v);
    const int lane = lin & 31, w = lin >> 5;
    if (lane == 0) ws[w] = v;
    __syncthreads();
    v = 0.0;
    if (w == 0) {
        v = lane < NT / 32 ? ws[lane] : 0.0;
        v = warp_sum(v);
    }
    return v;
}

// compensated accumulator: the exact value of the sum so far is s + c up to
// O(eps^2) relative terms.  The _rn intrinsics keep the compiler from fusing
// a product into a neighbouring add, which would break the error terms.
struct Acc2 {
    float s = 0.f, c = 0.f;
    // add the exact product x*y
    __device__ __forceinline__ void add_prod(float x, float y) {
        const float p = __fmul_rn(x, y);
        const float ep = fmaf(x, y, -p);  // TwoProduct error
        add(p, ep);
    }
    // add p + ep (ep a small correction)
    __device__ __forceinline__ void add(float p, float ep) {
        const float t = __fadd_rn(s, p);
        const float z = __fsub_rn(t, s);
        const float es = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));  // TwoSum error
        s = t;
        c = __fadd_rn(c, __fadd_rn(es, ep));
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

}  // namespace
}  // namespace claire
