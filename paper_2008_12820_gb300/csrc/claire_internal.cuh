// claire_internal.cuh -- internal declarations of the GB300 registration library.
//
// Layout (all device memory):
//   scalar field  float[n1][n2][n3]        (x3 contiguous)
//   vector field  float[3][n1][n2][n3]
//   half spectrum float2[c][n1][n2][p3]    (k3 = 0..h3-1 valid, h3 = n3/2+1,
//                                           p3 = h3 rounded up to 4: pitch)
// Wavenumbers on an axis of n points: index i -> i for 2i < n, else i - n.
// First derivatives use 0 at the Nyquist index of an even axis.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include <string>
#include <vector>

#include "claire.h"

namespace claire {

struct Profiler;

constexpr int kMaxStages = 16;
constexpr int kThreads = 256;

// plan of a 1D FFT of length n: radix per stage and the twiddle table
// tw[t] = exp(-2*pi*i*t/n), t = 0..n-1 (computed on the host in double)
struct FftPlan {
    int n;
    int nst;
    int rad[kMaxStages];
    const float2 *tw;
};

struct Dims {
    int n1, n2, n3;
    long long N;     // n1*n2*n3
    int h3, p3;      // half-spectrum length and pitch along x3
    int iorder = 3;  // interpolation of the SL steps: 3 cubic Lagrange, 1 trilinear
};

// spectral operators applied in the fused x1 pass
enum SpecOp { OP_GRAD = 0, OP_DIV = 1, OP_A = 2, OP_AINV = 3,
              // three components, x1 pass forward only / scale then inverse only
              OP_X1FWD = 4, OP_X1INV = 5 };

// epilogues of the inverse x3 pass
enum C2rEpi { EPI_STORE = 0, EPI_ADD = 1 };

struct SpecParams {
    float beta, gamma, scale;  // scale = 1/N folds the inverse-FFT normalization
};

// ------------------------------------------------------------------ FFT ----
// out-of-place forward: real [ncomp][n1][n2][n3] -> spectrum [ncomp] ;
// multiply ; inverse into real [nout][n1][n2][n3] (+ optional addend)
void spectral_apply(const Dims &d, const FftPlan *ax, SpecOp op, const SpecParams &sp,
                    const float *in, float *out, const float *add, float2 *spec,
                    cudaStream_t st, Profiler *prof);

// forward 3D transform of three components into spec (unnormalized), and the
// inverse from spec (scaled by sp.scale) into real fields; spec is consumed
void spectral_forward3(const Dims &d, const FftPlan *ax, const float *in, float2 *spec,
                       cudaStream_t st, Profiler *prof);
void spectral_inverse3(const Dims &d, const FftPlan *ax, float2 *spec, float *out, float scale,
                       cudaStream_t st, Profiler *prof);
// restriction of a fine half spectrum to a coarse grid (modes |k_d| < nc_d/2,
// times scale; others zero) for three components
void launch_spec_restrict(const Dims &df, const float2 *specf, const Dims &dc, float2 *specc,
                          float scale, cudaStream_t st, Profiler *prof);
// two-level combination on the fine spectrum, in place: modes the coarse grid
// holds take scale * coarse spectrum, the others become (beta0 A)^{-1} of
// themselves (the high-pass part of (beta0 A)^{-1} r)
void launch_spec_twolevel(const Dims &df, float2 *specf, const Dims &dc, const float2 *specc,
                          float scale, float beta0, float gamma, cudaStream_t st, Profiler *prof);

// eighth-order central finite differences (Section 4.2): gradient of a
// scalar field [N] -> [3][N], divergence of a vector field [3][N] -> [N]
void launch_grad_fd8(const Dims &d, const float *f, float *g, cudaStream_t st, Profiler *prof);
void launch_div_fd8(const Dims &d, const float *v, float *out, cudaStream_t st, Profiler *prof);

// ------------------------------------------------------------ transport ----
// Box entries: the SL kernels work on tiles of 32 (x3) x 8 (x2) x 4 (x1)
// voxels, ordered x3 fastest; a displacement field comes with one int4 per
// tile, {lo1, lo2, lo3, ok}: the smallest floor of the tile's displacements
// per axis, and whether all its floors fit the kernels' shared-memory box.
long long tile_count(const Dims &d);
// Foot points and the box entries of each output (tile_count(d) int4 each).
// Either of dispm (X-) and dispp (X+) may be null; that side is skipped.
void launch_footpoints(const Dims &d, int nt, const float *v, float *dispm, float *dispp, int4 *tiles_m,
                       int4 *tiles_p, cudaStream_t st, Profiler *prof);
// box entries of an arbitrary displacement field
void launch_tile_ranges(const Dims &d, const float *disp, int4 *tiles, cudaStream_t st, Profiler *prof);
void launch_interp(const Dims &d, const float *f, const float *disp, float *out, int4 *tiles,
                   cudaStream_t st, Profiler *prof, int kclass);
void launch_adjoint_factor(const Dims &d, int nt, const float *divv, const float *dispp,
                           const int4 *tiles_p, float *cfac, cudaStream_t st, Profiler *prof);
// dst_h (optional): an FP16 copy of dst, the stored trajectory of the
// FP16-storage form
void launch_state_step(const Dims &d, const float *src, const float *dispm, const int4 *tiles_m,
                       float *dst, cudaStream_t st, Profiler *prof, __half *dst_h = nullptr);
void launch_adjoint_step(const Dims &d, const float *src, const float *dispp, const int4 *tiles_p,
                         const float *cfac, float *dst, cudaStream_t st, Profiler *prof, int kclass,
                         __half *dst_h = nullptr);
void launch_incstate_init(const Dims &d, float dt, const float *vt, const float *gm0, float *u0,
                          cudaStream_t st, Profiler *prof);
void launch_incstate_step(const Dims &d, float dt, const float *src, const float *dispm,
                          const int4 *tiles_m, const float *vt, const float *gm_next, float *dst,
                          cudaStream_t st, Profiler *prof);
// the last incremental-state step fused with the incremental adjoint's final
// condition: lt_last = -mt(1), mt_out (nullable) = mt(1), b_out (nullable)
// [3][N] = the body force's first term dt/2 lt(1) grad m(1)
void launch_incstate_last(const Dims &d, float dt, const float *src, const float *dispm, const int4 *tiles_m,
                          const float *vt, const float *gm_last, float *lt_last, float *mt_out, float *b_out,
                          cudaStream_t st, Profiler *prof);
void launch_incstate_last(const Dims &d, float dt, const float *src, const float *dispm, const int4 *tiles_m,
                          const float *vt, const __half *gm_last, float *lt_last, float *mt_out, float *b_out,
                          cudaStream_t st, Profiler *prof);
// adjoint step dst = c src(X+) that also adds w dst grad m^{j-1} to the body
// force b [3][N] in place (gm = grad m^{j-1}).  With want_dot it also forms
// p . b of the updated b (b . b if p is null): block partials in partial,
// their sum plus *dot_add (nullable) in *dot_out.  dst_h: optional FP16 copy
// of dst.
void launch_adjoint_acc(const Dims &d, const float *src, const float *dispp, const int4 *tiles_p, const float *cfac,
                        float *dst, const float *gm, float *b, float w, bool want_dot, const float *p,
                        double *partial, const double *dot_add, double *dot_out, cudaStream_t st, Profiler *prof,
                        int kclass, __half *dst_h = nullptr);
void launch_adjoint_acc(const Dims &d, const float *src, const float *dispp, const int4 *tiles_p, const float *cfac,
                        float *dst, const __half *gm, float *b, float w, bool want_dot, const float *p,
                        double *partial, const double *dot_add, double *dot_out, cudaStream_t st, Profiler *prof,
                        int kclass, __half *dst_h = nullptr);
// the adjoint's final condition l = m1 - m (l_h: optional FP16 copy) and the
// gradient started as g = Av + w l gm  (gm = grad m(1), w = dt/2)
void launch_adjfinal_acc(const Dims &d, const float *m1, const float *m, float *l, __half *l_h, const float *gm,
                         const float *Av, float *g, float w, cudaStream_t st, Profiler *prof);
void launch_adjfinal_acc(const Dims &d, const float *m1, const float *m, float *l, __half *l_h, const __half *gm,
                         const float *Av, float *g, float w, cudaStream_t st, Profiler *prof);
// b += w * l * gm
void launch_bodyforce_acc(const Dims &d, float *b, const float *l, const float *gm, float w,
                          cudaStream_t st, Profiler *prof);
// l = gmis * (m1 - m) - gm_final * inv_h3 (gm_final nullable)
void launch_adjoint_final(const Dims &d, float *l, const float *m1, const float *m,
                          const float *gm_final, float gmis, float inv_h3, cudaStream_t st,
                          Profiler *prof);

// FP16-storage form: the stored trajectories (m^j, grad m^j, lambda^j) are
// FP16; these overloads read them as such and compute in FP32
void launch_incstate_init(const Dims &d, float dt, const float *vt, const __half *gm0, float *u0,
                          cudaStream_t st, Profiler *prof);
void launch_incstate_step(const Dims &d, float dt, const float *src, const float *dispm,
                          const int4 *tiles_m, const float *vt, const __half *gm_next, float *dst,
                          cudaStream_t st, Profiler *prof);
// FP16 <-> FP32 copies of n values
void launch_f2h(const float *in, __half *out, long long n, cudaStream_t st, Profiler *prof);
void launch_h2f(const __half *in, float *out, long long n, cudaStream_t st, Profiler *prof);
// spectral gradient / divergence by axis transforms: d/dx_a = F_a^-1 i k^_a F_a
// (the same operator as through the 3D transform, one pass per axis)
void spectral_grad_1d(const Dims &d, const FftPlan *ax, const float *f, float *g, cudaStream_t st, Profiler *prof);
void spectral_grad_1d(const Dims &d, const FftPlan *ax, const float *f, __half *g, cudaStream_t st, Profiler *prof);
void spectral_div_1d(const Dims &d, const FftPlan *ax, const float *v, float *out, cudaStream_t st, Profiler *prof);
void launch_grad_fd8(const Dims &d, const float *f, __half *g, cudaStream_t st, Profiler *prof);

// ------------------------------------------------------------- vectors ----
// FP64 reductions; results land in dev_out[0..k) (device doubles)
// dev_out[0] = sum of partial[0..nb) (+ add[0] if add is non-null)
void launch_finalize(const double *partial, int nb, const double *add, double *dev_out, cudaStream_t st);
// the four dot products of the line search: dev_out[0..3] = g.x, x.Av, v.Ax, x.Ax
void launch_ls_dots(const float *g, const float *x, const float *Av, const float *v, const float *Ax, long long n,
                    double *partial, double *dev_out, cudaStream_t st, Profiler *prof);
void launch_dot(const float *a, const float *b, long long n, double *partial, double *dev_out,
                cudaStream_t st, Profiler *prof);
void launch_sqdiff(const float *a, const float *b, long long n, double *partial,
                   double *dev_out, cudaStream_t st, Profiler *prof);
void launch_pcg_xr(float *x, float *r, const float *p, const float *q, float alpha,
                   long long n, double *partial, double *dev_out, cudaStream_t st,
                   Profiler *prof);  // x += a p, r -= a q, out = ||r||^2
void launch_pcg_p(float *p, const float *z, float beta, long long n, cudaStream_t st,
                  Profiler *prof);   // p = z + beta p
void launch_axpby(float *out, float a, const float *x, float b, const float *y, long long n,
                  cudaStream_t st, Profiler *prof);  // out = a x + b y
void launch_diff_flag(const float *a, const float *b, long long n, int *flag, cudaStream_t st,
                      Profiler *prof);
// stats of a vector field [3][N]: dev_out[0] = r.r, dev_out[1..3] = component sums
void launch_stats(const float *r, long long N, double *partial, double *dev_out, cudaStream_t st,
                  Profiler *prof);
// x += a p; Ax += a Ap; r -= a q (q_adds_Ap: r -= a (q + Ap), q holding the
// body force of H p only); then the stats of r into dev_out[0..3]
void launch_pcg_update(float *x, float *Ax, float *r, const float *p, const float *Ap,
                       const float *q, float alpha, long long N, double *partial, double *dev_out,
                       cudaStream_t st, Profiler *prof, bool q_adds_Ap = false, const double *dpq = nullptr,
                       const double *drz = nullptr, double *pq_out = nullptr);
// p = z + b p; Ap = (r - mean r) + b Ap (rsum: device component sums of r);
// with Az given (beta*A z), Ap = Az + b Ap instead.  x += a p skips Ax if NULL.
void launch_pcg_dir(float *p, float *Ap, const float *z, const float *r, const double *rsum,
                    const float *Az, float b, long long N, bool init, cudaStream_t st,
                    Profiler *prof, const double *dbn = nullptr, const double *dbd = nullptr);
// device-side control of the inner PCG of the H0 preconditioners (a CUDA
// graph with a conditional while node; the control kernel sets the loop's
// condition and that of the IF node around the rest of the body, h_tail);
// c: the loop's device scalars,
// c[0] tolerance, c[1] ||r0||, c[2] p.q, c[3] r.z (current direction),
// c[4] r.z (new residual), c[5] iterations, c[6..9] stats of r, c[10] bodies
void launch_inner_init(double *c, cudaStream_t st, Profiler *prof);
void launch_inner_ctl(double *c, cudaGraphConditionalHandle h, cudaGraphConditionalHandle h_tail, int maxit,
                      bool fixed, cudaStream_t st, Profiler *prof);
void launch_scalar_copy(double *dst, const double *src, cudaStream_t st, Profiler *prof);
// device-side control of the outer PCG loop (InvA) as a graph: k_pcg_ctl
// reads d[0] (||r||^2) and d[12] (p.Hp) of the solver's result slots and
// keeps c[0] threshold, c[1] iterations, c[2] flags, c[3] bodies
void launch_pcg_ctl(const double *d, double *c, cudaGraphConditionalHandle h, cudaGraphConditionalHandle h_tail,
                    int maxit, bool fixed, cudaStream_t st, Profiler *prof);
void launch_pcg_negcopy(const double *c, float *x, float *Ax, const float *z, const float *Ap, long long n,
                        cudaStream_t st, Profiler *prof);
void launch_pcg_ctl_init(double *c, double thr, cudaStream_t st, Profiler *prof);
void launch_scalar_set(double *dst, double v, cudaStream_t st, Profiler *prof);
// launch_pcg_dir that also writes u0 = dt/2 * (-p . gm0) (N floats), the
// first incremental-state field of the next matvec (hdt = dt/2), and, with
// pap_out non-null, p . Ap of the new direction into *pap_out
void launch_pcg_dir_u0(float *p, float *Ap, const float *z, const float *r, const double *rsum, const float *Az,
                       float b, long long N, bool init, const float *gm0, float *u0, float hdt, double *partial,
                       double *pap_out, cudaStream_t st, Profiler *prof, const double *dbn = nullptr,
                       const double *dbd = nullptr);
void launch_pcg_dir_u0(float *p, float *Ap, const float *z, const float *r, const double *rsum, const float *Az,
                       float b, long long N, bool init, const __half *gm0, float *u0, float hdt, double *partial,
                       double *pap_out, cudaStream_t st, Profiler *prof, const double *dbn = nullptr,
                       const double *dbd = nullptr);
// q = Ap + gm (gm . p): the zero-velocity Hessian given beta0*A p
void launch_h0_apply(float *q, const float *Ap, const float *gm, const float *p, long long N,
                     cudaStream_t st, Profiler *prof);
constexpr int kReduceBlocks = 1216;  // 152 SMs x 8

// grid of a persistent transform pass: as many blocks as fit the SMs at this
// shared memory per block (227 KB per SM, 1 KB reserved per block, at most 8
// per SM), at most nitems
int persistent_grid(long long nitems, size_t smem);

// ------------------------------------------------- kernel attributes ----
// Reports a failed cudaFuncSetAttribute as a library error with the kernel's
// name (thrown to the ABI call that launched it; defined in capi.cu).
[[noreturn]] void attr_failed(const char *kernel, cudaError_t e);

// A kernel's dynamic shared-memory limit above the 48 KB default, raised per
// device: the attribute belongs to the device's context, so a context on
// another device needs its own call.  The largest limit set so far is kept
// per device (kernels with a runtime-sized plan ask for different sizes), so
// steady-state launches make no runtime call.  Thread-safe; a failure is
// reported with the kernel's name instead of surfacing later as a failed
// launch.
struct SmemAttr {
    static constexpr int kDevices = 64;
    std::atomic<int> set[kDevices] = {};  // bytes set so far, per device index
    template <typename K>
    void ensure(K kernel, int bytes, const char *name) {
        if (bytes <= 48 * 1024) return;
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) attr_failed(name, e);
        std::atomic<int> *slot = dev >= 0 && dev < kDevices ? &set[dev] : nullptr;
        if (slot && slot->load(std::memory_order_acquire) >= bytes) return;
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            attr_failed(name, e);
        }
        if (slot) {
            int cur = slot->load(std::memory_order_acquire);
            while (cur < bytes && !slot->compare_exchange_weak(cur, bytes, std::memory_order_acq_rel)) {
            }
        }
    }
};

// ------------------------------------------------------------ profiler ----
// Counts kernel launches and, when on, brackets each launch group with CUDA
// events on its stream and records the algorithmic HBM bytes it moves (each
// input and output field counted once, gathers counted as one read).
struct Profiler {
    bool on = false;
    long launches = 0;
    struct Rec { cudaEvent_t a, b; int cls; double bytes; };
    std::vector<Rec> recs;
    size_t used = 0;
    // mark the start of a launch of class cls on stream st; returns slot or -1
    int begin(int cls, double bytes, cudaStream_t st);
    void end(int slot, cudaStream_t st);
    void reset();
    ~Profiler();
};

struct ProfScope {
    Profiler *p;
    int slot;
    cudaStream_t st;
    // nk = kernels launched inside the scope
    ProfScope(Profiler *p_, int cls, cudaStream_t st_, double bytes = 0, int nk = 1)
        : p(p_), slot(-1), st(st_) {
        if (p) { p->launches += nk; slot = p->begin(cls, bytes, st); }
    }
    ~ProfScope() { if (p && slot >= 0) p->end(slot, st); }
};

}  // namespace claire
