// noalloc.cu -- claire_precond_noalloc: the spectral preconditioner
// s = (beta*A)^{-1} r without any device allocation.
//
// Some callers cannot allocate device memory at all: code running under a
// host framework that owns the whole device heap (a fixed arena carved out at
// start-up), code that must not call cudaMalloc/cudaFree because they
// synchronize the device, or a caller that has to stay within a memory budget
// it cannot grow.  They still hold their own input and output buffers.  For
// them this entry point keeps its scratch (the half spectrum of the three
// components and the FFT twiddle tables) in file-scope device arrays that
// every GPU loading the library holds until the process exits.
//
// Host code sees those arrays only through host-side stand-ins; their device
// addresses come from cudaGetSymbolAddress, looked up once per device with
// that device current (the first call on a device does it, so that first
// call should come before any stream capture).  The addresses are kept for
// the life of the process, so a device reset after that first call is not
// supported (the module's arrays could then sit elsewhere).  All calls on a
// device share
// the arrays: calls whose work overlaps on the GPU (different streams, or
// several host threads) race on them and must be serialized by the caller.
// The arrays keep the last call's contents; nothing in them needs to start at
// zero, because every spectrum entry a call reads it has written before.
#include <cuda_runtime.h>

#include <cmath>
#include <exception>
#include <mutex>
#include <string>

#include "claire.h"
#include "claire_internal.cuh"

namespace claire {
void set_thread_error(const std::string &msg);  // capi.cu
}

namespace {

using namespace claire;

// scratch capacity: half spectra of three components, 3 * nx * ny * p3 complex
// values with p3 = (nz/2 + 1) rounded up to 4; 442368 covers a 64^3 grid
constexpr long long kSpecCap = 442368;
constexpr int kMaxAxis = 1024;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float2 g_spec[kSpecCap];
static __device__ __align__(256) float2 g_tw[3 * kMaxAxis];

struct DevScratch {
    float2 *spec = nullptr;
    float2 *tw = nullptr;
};
DevScratch g_scratch[kMaxDevices];
std::mutex g_mu;

// twiddle table tw[t] = exp(-2 pi i t / n), evaluated in double
__global__ void k_twiddles(float2 *tw, int n) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) {
        double c, s;
        sincospi(2.0 * (double)t / (double)n, &s, &c);
        tw[t] = make_float2((float)c, (float)(-s));
    }
}

bool axis_ok(int n) {
    if (n < 4 || n > kMaxAxis) return false;
    for (int p : {2, 3, 5})
        while (n % p == 0) n /= p;
    return n == 1;
}

FftPlan axis_plan(int n, const float2 *tw) {
    FftPlan p{};
    p.n = n;
    p.tw = tw;
    int m = n;
    while (m % 4 == 0) { p.rad[p.nst++] = 4; m /= 4; }
    while (m % 2 == 0) { p.rad[p.nst++] = 2; m /= 2; }
    while (m % 3 == 0) { p.rad[p.nst++] = 3; m /= 3; }
    while (m % 5 == 0) { p.rad[p.nst++] = 5; m /= 5; }
    return p;
}

int fail(int code, const std::string &msg) {
    set_thread_error(msg);
    return code;
}

}  // namespace

extern "C" int claire_precond_noalloc(int nx, int ny, int nz, double beta, double gamma,
                                      const float *r, float *s, void *stream) {
    if (!r || !s) return fail(CLAIRE_ERR_ARG, "claire_precond_noalloc: r and s must not be NULL");
    if (!axis_ok(nx) || !axis_ok(ny) || !axis_ok(nz))
        return fail(CLAIRE_ERR_ARG,
                    "claire_precond_noalloc: grid sizes must be in [4, 1024] with prime factors 2, 3, 5");
    if (!(beta > 0) || !std::isfinite(beta) || !(gamma >= 0) || !std::isfinite(gamma))
        return fail(CLAIRE_ERR_ARG, "claire_precond_noalloc: need beta > 0 and gamma >= 0, finite");
    Dims d{};
    d.n1 = nx;
    d.n2 = ny;
    d.n3 = nz;
    d.N = (long long)nx * ny * nz;
    d.h3 = nz / 2 + 1;
    d.p3 = (d.h3 + 3) / 4 * 4;
    const long long need = 3LL * nx * ny * d.p3;
    if (need > kSpecCap)
        return fail(CLAIRE_ERR_ARG,
                    "claire_precond_noalloc: grid too large for the built-in scratch (needs " +
                        std::to_string(need) + " complex values, capacity " +
                        std::to_string(kSpecCap) + ", e.g. 64^3)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(CLAIRE_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(CLAIRE_ERR_ARG, "claire_precond_noalloc: device index too large");
    DevScratch sc;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch[dev].spec) {
            // one-time set-up on this device (it is current): device addresses
            // of the file-scope arrays
            void *ps = nullptr, *pt = nullptr;
            e = cudaGetSymbolAddress(&ps, g_spec);
            if (e != cudaSuccess)
                return fail(CLAIRE_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            e = cudaGetSymbolAddress(&pt, g_tw);
            if (e != cudaSuccess)
                return fail(CLAIRE_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_scratch[dev].spec = (float2 *)ps;
            g_scratch[dev].tw = (float2 *)pt;
        }
        sc = g_scratch[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int ns[3] = {nx, ny, nz};
    FftPlan ax[3];
    for (int a = 0; a < 3; ++a) {
        float2 *tw = sc.tw + a * kMaxAxis;
        k_twiddles<<<(ns[a] + 127) / 128, 128, 0, st>>>(tw, ns[a]);
        ax[a] = axis_plan(ns[a], tw);
    }
    const SpecParams sp{(float)beta, (float)gamma, (float)(1.0 / (double)d.N)};
    try {
        spectral_apply(d, ax, OP_AINV, sp, r, s, nullptr, sc.spec, st, nullptr);
    } catch (const std::exception &ex) {
        return fail(CLAIRE_ERR_CUDA, std::string("claire_precond_noalloc: ") + ex.what());
    }
    e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(CLAIRE_ERR_CUDA, std::string("claire_precond_noalloc: ") + cudaGetErrorString(e));
    }
    return CLAIRE_OK;
}
