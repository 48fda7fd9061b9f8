// capi.cu -- the C ABI (include/claire.h): context and workspace, the
// linearization cache, reduced gradient (Eq. 3.1), Gauss-Newton Hessian matvec
// (Eq. 3.4), spectral preconditioner, PCG and the Gauss-Newton-Krylov solver
// with Armijo line search (Algorithm 1, Eq. 3.3).
//
// All arithmetic on fields runs in the kernels of transport.cu, fft.cu and
// vec.cu; this file only sequences launches on the context's stream and reads
// back the FP64 scalars the Krylov and Newton iterations branch on.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <exception>
#include <new>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include <algorithm>
#include <atomic>

#include <nvtx3/nvToolsExt.h>

#include "claire.h"
#include "claire_internal.cuh"

using namespace claire;

namespace {

struct Error : std::exception {
    int code;
    std::string msg;
    Error(int c, std::string m) : code(c), msg(std::move(m)) {}
    const char *what() const noexcept override { return msg.c_str(); }
};

void check_cuda(cudaError_t e, const char *what) {
    if (e != cudaSuccess) {
        cudaGetLastError();  // clear a non-sticky error so the context stays usable
        throw Error(e == cudaErrorMemoryAllocation ? CLAIRE_ERR_OOM : CLAIRE_ERR_CUDA,
                    std::string(what) + ": " + cudaGetErrorString(e));
    }
}
#define CK(x) check_cuda((x), #x)

void check_launch(const char *where) {
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error(CLAIRE_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
    }
}

thread_local std::string g_create_error = "no error";
// process-wide cap on the device bytes one context may allocate (0: none)
std::atomic<size_t> g_workspace_limit{0};

bool valid_n(int n) {
    if (n < 4 || n > 1024) return false;
    for (int p : {2, 3, 5})
        while (n % p == 0) n /= p;
    return n == 1;
}

// radix sequence for a length-n Stockham FFT: 4s first, then 2, 3, 5
FftPlan make_plan(int n) {
    FftPlan p{};
    p.n = n;
    int m = n;
    while (m % 4 == 0) { p.rad[p.nst++] = 4; m /= 4; }
    while (m % 2 == 0) { p.rad[p.nst++] = 2; m /= 2; }
    while (m % 3 == 0) { p.rad[p.nst++] = 3; m /= 3; }
    while (m % 5 == 0) { p.rad[p.nst++] = 5; m /= 5; }
    return p;
}

}  // namespace

// ------------------------------------------------------------- profiler ----
namespace claire {
// message returned by claire_last_error(NULL) on this thread
void set_thread_error(const std::string &msg) { g_create_error = msg; }

void attr_failed(const char *kernel, cudaError_t e) {
    throw Error(CLAIRE_ERR_CUDA, std::string("cudaFuncSetAttribute (dynamic shared memory) of ") + kernel + ": " +
                                     cudaGetErrorString(e));
}

int Profiler::begin(int cls, double bytes, cudaStream_t st) {
    if (!on) return -1;
    if (used == recs.size()) {
        Rec r{};
        if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) return -1;
        recs.push_back(r);
    }
    recs[used].cls = cls;
    recs[used].bytes = bytes;
    cudaEventRecord(recs[used].a, st);
    return (int)used++;
}
void Profiler::end(int slot, cudaStream_t st) { cudaEventRecord(recs[slot].b, st); }
void Profiler::reset() { used = 0; }
Profiler::~Profiler() {
    for (auto &r : recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
}
}  // namespace claire

// --------------------------------------------------------------- context ---
struct claire_ctx {
    Dims d{};
    int nt = 0;
    double beta = 0, gamma = 0;
    cudaStream_t st = 0;
    std::string err = "no error";
    FftPlan ax[3]{};
    Profiler prof;
    std::vector<void *> allocs;
    size_t bytes = 0;

    float *m0 = nullptr, *m1 = nullptr;
    float *vlin = nullptr, *dispm = nullptr, *dispp = nullptr;
    float *mhist = nullptr, *gmhist = nullptr, *divv = nullptr, *cfac = nullptr;
    float *lhist = nullptr, *mt = nullptr;
    // FP16-storage form: the state trajectory m^j, its gradient grad m^j and
    // the gradient's adjoint lambda^j are stored in FP16.  The transport itself
    // runs in FP32 (two scratch fields in turn, each step also writing the FP16
    // copy), grad m^j is taken of the FP32 state before it is rounded, and the
    // final state m(1) is kept in FP32 (m1f) for the mismatch and lambda(1).
    // The incremental fields of the matvec stay FP32 (their scale follows the
    // PCG direction); gm1f holds grad m(1) in FP32 for the H0 preconditioners.
    bool h16 = false;
    __half *mhist_h = nullptr, *gmhist_h = nullptr, *lhist_h = nullptr;
    float *gm1f = nullptr, *m1f = nullptr;
    float *s3a = nullptr, *s1a = nullptr, *s1b = nullptr, *fdisp = nullptr;
    float2 *spec = nullptr;
    double *partial = nullptr, *dres = nullptr;
    int *dflag = nullptr;
    // box entries (one int4 per transport tile) of the displacement fields:
    // X-, X+, forward-only X-, interp (the X- and forward-only slots swap when
    // a line-search trial is adopted)
    int4 *rng = nullptr;
    long long ntiles = 0;
    int off_m = 0, off_f = 2;
    int4 *rng_m() { return rng + off_m * ntiles; }
    int4 *rng_p() { return rng + 1 * ntiles; }
    int4 *rng_f() { return rng + off_f * ntiles; }
    int4 *rng_i() { return rng + 3 * ntiles; }
    // solver vectors, allocated on the first solve
    float *sv = nullptr;
    // state history of the line search's trial velocity (solver only): an
    // accepted trial becomes the next linearization's state as it stands
    float *mhist_t = nullptr;

    bool have_images = false, have_lin = false;
    // host-buffer solves (claire_solve_host): a second stream copies the
    // images in while the first foot points run, and v out while the final
    // gradient runs; vdev holds v on the device
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_main = nullptr, ev_img = nullptr, ev_vout = nullptr;
    bool img_pending = false;  // the image copies on aux may still be running
    float *vdev = nullptr;
    void ensure_aux() {
        if (aux) return;
        CK(cudaStreamCreateWithFlags(&aux, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&ev_main, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ev_img, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ev_vout, cudaEventDisableTiming));
    }
    // order the main stream after the image copies (before m0 or m1 is read)
    void wait_images() {
        if (img_pending) {
            CK(cudaStreamWaitEvent(st, ev_img, 0));
            img_pending = false;
        }
    }
    // grad m^0 = grad m0 in gmhist slot 0 is current (m0 and the derivative
    // scheme unchanged since it was computed; a solve recomputes it once)
    bool gm0_valid = false;
    bool deriv_fd8 = false;  // first derivatives by FD8 instead of spectral
    double last_vAv = 0;  // <v, beta A v> (grid sum) of the last gradient with J

    float *alloc_f(size_t n) { return (float *)alloc_bytes(n * sizeof(float)); }
    __half *alloc_h(size_t n) { return (__half *)alloc_bytes(n * sizeof(__half)); }
    void *alloc_bytes(size_t b) {
        const size_t cap = g_workspace_limit.load();
        if (cap && bytes + b > cap)
            throw Error(CLAIRE_ERR_OOM, "workspace limit of " + std::to_string(cap) + " bytes: the context holds " +
                                            std::to_string(bytes) + " and needs " + std::to_string(b) + " more");
        void *p = nullptr;
        CK(cudaMalloc(&p, b));
        allocs.push_back(p);
        bytes += b;
        return p;
    }
    // free what was allocated after a mark (a lazy allocation group that
    // failed part way: its members are only assigned once all succeeded)
    void rollback(size_t mark, size_t bytes0) {
        while (allocs.size() > mark) {
            cudaFree(allocs.back());
            allocs.pop_back();
        }
        bytes = bytes0;
    }
    ~claire_ctx() {
        if (mvg.exec) cudaGraphExecDestroy(mvg.exec);
        drop_inner_graphs();
        drop_pcg_graphs();
        if (side) {
            cudaStreamSynchronize(side);
            cudaStreamDestroy(side);
            cudaEventDestroy(ev_fork);
            cudaEventDestroy(ev_join);
        }
        if (aux) {
            cudaStreamSynchronize(aux);
            cudaStreamDestroy(aux);
            cudaEventDestroy(ev_main);
            cudaEventDestroy(ev_img);
            cudaEventDestroy(ev_vout);
        }
        for (void *p : allocs) cudaFree(p);
        for (int a = 0; a < 3; ++a) cudaFree((void *)ax[a].tw);
    }

    long long N() const { return d.N; }
    float *hist(float *base, int j, int comps = 1) const { return base + (size_t)j * comps * d.N; }
    __half *hist(__half *base, int j, int comps = 1) const { return base + (size_t)j * comps * d.N; }
    // grad m(1) of the linearization in FP32
    const float *gm_final() { return h16 ? gm1f : hist(gmhist, nt, 3); }
    double h3() const {
        const double tp = 6.283185307179586476925286766559;
        return (tp / d.n1) * (tp / d.n2) * (tp / d.n3);
    }
    SpecParams sp(double b = -1) const {
        return SpecParams{(float)(b > 0 ? b : beta), (float)gamma, (float)(1.0 / (double)d.N)};
    }
    // beta inside the zero-velocity Hessian H0 (Section 3 "Preconditioning":
    // floored at 5e-2 so the preconditioner stays effective for small beta)
    double beta_h0() const { return beta < 5e-2 ? 5e-2 : beta; }
    float *ih = nullptr;  // inner PCG vectors: r, z, p, q, Ap (5 x 3N)

    double fetch(int slot = 0) {
        double h = 0;
        fetch_n(slot, 1, &h);
        return h;
    }
    void fetch_n(int slot, int n, double *h) {
        CK(cudaMemcpyAsync(h, dres + slot, n * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    double dot(const float *a, const float *b, long long n) {
        launch_dot(a, b, n, partial, dres, st, &prof);
        return fetch();
    }

    // ---- operators ------------------------------------------------------
    void spectral(SpecOp op, const float *in, float *out, const float *add, double b = -1) {
        spectral_apply(d, ax, op, sp(b), in, out, add, spec, st, &prof);
    }

    // FFT resources of one grid (the context's grid, or its half-resolution
    // grid for the two-level preconditioner)
    struct Grid {
        Dims d{};
        const FftPlan *ax = nullptr;
        float2 *spec = nullptr;
    };
    Grid fine() const { return Grid{d, ax, spec}; }

    // half-resolution grid of the two-level preconditioner, made on first use
    struct Coarse {
        Dims d{};
        FftPlan ax[3]{};
        float2 *spec = nullptr;
        float *gm = nullptr, *r = nullptr, *s = nullptr, *work = nullptr;
        bool gm_valid = false;
        bool ready = false;
    } co;

    void make_coarse() {
        if (co.ready) return;
        const int ns[3] = {d.n1 / 2, d.n2 / 2, d.n3 / 2};
        for (int a = 0; a < 3; ++a)
            if ((2 * ns[a] != (a == 0 ? d.n1 : a == 1 ? d.n2 : d.n3)) || !valid_n(ns[a]))
                throw Error(CLAIRE_ERR_ARG, "two-level preconditioner needs even grid sizes >= 8 whose halves are valid FFT lengths");
        co.d.n1 = ns[0];
        co.d.n2 = ns[1];
        co.d.n3 = ns[2];
        co.d.N = (long long)ns[0] * ns[1] * ns[2];
        co.d.h3 = ns[2] / 2 + 1;
        co.d.p3 = (co.d.h3 + 3) / 4 * 4;
        for (int a = 0; a < 3; ++a) {
            co.ax[a] = make_plan(ns[a]);
            std::vector<float2> tw(ns[a]);
            for (int t = 0; t < ns[a]; ++t) {
                const double ang = 6.283185307179586476925286766559 * (double)t / (double)ns[a];
                tw[t] = make_float2((float)std::cos(ang), (float)(-std::sin(ang)));
            }
            float2 *dtw = (float2 *)alloc_bytes(ns[a] * sizeof(float2));
            CK(cudaMemcpy(dtw, tw.data(), ns[a] * sizeof(float2), cudaMemcpyHostToDevice));
            co.ax[a].tw = dtw;
        }
        const size_t Nc = co.d.N;
        co.spec = (float2 *)alloc_bytes((size_t)3 * ns[0] * ns[1] * co.d.p3 * sizeof(float2));
        co.gm = alloc_f(3 * Nc);
        co.r = alloc_f(3 * Nc);
        co.s = alloc_f(3 * Nc);
        co.work = alloc_f(15 * Nc);
        co.ready = true;
    }

    // s = H0^{-1} r on grid g by PCG preconditioned with (beta0 A)^{-1},
    // x0 = 0, stop at ||r_i|| <= tol ||r_0|| (or after exactly maxit
    // iterations if fixed); H0 = beta0 A + gm (x) gm.  beta0 A p is carried by
    // the same recurrence as in the outer PCG.  work: 5 vectors of g.  Uses
    // result slots dres[4..7] so the caller's residual sums survive.
    // ---- loops as CUDA graphs ---------------------------------------------
    // Builds [setup] -> WHILE(hw) { head ; IF(hif) { tail } } and instantiates
    // it.  head ends with a control kernel that sets both conditions (the
    // loop's and the tail's) to "continue": the tail -- preconditioner and next
    // direction -- runs only when another iteration follows.  setup, head and
    // tail launch onto the context's stream, which is being captured.  The
    // kernels each part launches are returned (k_setup, k_head, k_tail).
    // false if the runtime refused (nothing has run).
    template <typename FS, typename FH, typename FT>
    bool build_loop_graph(cudaGraphExec_t *exec, FS &&setup, bool has_setup, FH &&head, FT &&tail, long &k_setup,
                          long &k_head, long &k_tail) {
        *exec = nullptr;
        const long k0 = prof.launches;
        k_setup = k_head = k_tail = 0;
        cudaGraph_t G = nullptr;
        cudaGraphConditionalHandle hw = 0, hif = 0;
        bool ok = cudaGraphCreate(&G, 0) == cudaSuccess &&
                  cudaGraphConditionalHandleCreate(&hw, G, 1, cudaGraphCondAssignDefault) == cudaSuccess;
        // captures fn into graph `into` (a fresh graph if null); returns it
        auto capture = [&](cudaGraph_t into, auto &&fn, cudaGraph_t *fresh) -> bool {
            const cudaError_t e0 = into ? cudaStreamBeginCaptureToGraph(st, into, nullptr, nullptr, 0,
                                                                        cudaStreamCaptureModeThreadLocal)
                                        : cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
            if (e0 != cudaSuccess) return false;
            try {
                fn();
            } catch (...) {
                cudaGraph_t tmp = nullptr;
                cudaStreamEndCapture(st, &tmp);
                if (tmp && !into) cudaGraphDestroy(tmp);
                if (G) cudaGraphDestroy(G);
                prof.launches = k0;
                throw;
            }
            cudaGraph_t out = nullptr;
            if (cudaStreamEndCapture(st, &out) != cudaSuccess || !out) return false;
            if (fresh) *fresh = out;
            return true;
        };
        cudaGraphNode_t nsetup = nullptr;
        if (ok && has_setup) {
            cudaGraph_t gi = nullptr;
            long ka = prof.launches;
            ok = capture(nullptr, setup, &gi);
            k_setup = prof.launches - ka;
            if (ok) ok = cudaGraphAddChildGraphNode(&nsetup, G, nullptr, 0, gi) == cudaSuccess;
            if (gi) cudaGraphDestroy(gi);
        }
        cudaGraphNodeParams cw = {};
        cudaGraphNode_t nw = nullptr;
        if (ok) {
            cw.type = cudaGraphNodeTypeConditional;
            cw.conditional.handle = hw;
            cw.conditional.type = cudaGraphCondTypeWhile;
            cw.conditional.size = 1;
            ok = cudaGraphAddNode(&nw, G, nsetup ? &nsetup : nullptr, nullptr, nsetup ? 1 : 0, &cw) == cudaSuccess;
        }
        cudaGraph_t body = ok ? cw.conditional.phGraph_out[0] : nullptr;
        if (ok) ok = cudaGraphConditionalHandleCreate(&hif, body, 0, 0) == cudaSuccess;
        cudaGraph_t tailg = nullptr;
        if (ok) {
            // the head, then the IF node behind its last node (added to the
            // graph being captured, the capture continuing from it)
            long ka = prof.launches;
            ok = capture(body, [&] {
                head(hw, hif);
                cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
                const cudaGraphNode_t *deps = nullptr;
                size_t nd = 0;
                cudaGraph_t cg = nullptr;
                bool ok2 = cudaStreamGetCaptureInfo(st, &cs, nullptr, &cg, &deps, nullptr, &nd) == cudaSuccess &&
                           cs == cudaStreamCaptureStatusActive;
                cudaGraphNodeParams ci = {};
                cudaGraphNode_t nif = nullptr;
                if (ok2) {
                    ci.type = cudaGraphNodeTypeConditional;
                    ci.conditional.handle = hif;
                    ci.conditional.type = cudaGraphCondTypeIf;
                    ci.conditional.size = 1;
                    ok2 = cudaGraphAddNode(&nif, cg, deps, nullptr, nd, &ci) == cudaSuccess;
                }
                if (ok2)
                    ok2 = cudaStreamUpdateCaptureDependencies(st, &nif, nullptr, 1, cudaStreamSetCaptureDependencies) ==
                          cudaSuccess;
                if (ok2) tailg = ci.conditional.phGraph_out[0];
            }, nullptr);
            k_head = prof.launches - ka;
            ok = ok && tailg;
        }
        if (ok) {
            long ka = prof.launches;
            ok = capture(tailg, tail, nullptr);
            k_tail = prof.launches - ka;
        }
        prof.launches = k0;
        if (ok) ok = cudaGraphInstantiate(exec, G, 0) == cudaSuccess;
        if (G) cudaGraphDestroy(G);
        if (!ok) {
            cudaGetLastError();
            *exec = nullptr;
        }
        return ok;
    }

    // The inner PCG as one CUDA graph: the setup (s = 0, r, ||r0||, the first
    // preconditioned direction) and a conditional WHILE node whose body is one
    // PCG iteration.  Step length, direction ratio and the stopping test are
    // evaluated on the device in the same FP64 arithmetic as the host-driven
    // loop below (same iterates and counts), so an inner solve costs one graph
    // launch and one host read instead of three round trips per iteration.
    // The executable graph is cached per grid and buffer set; the tolerance
    // goes through device memory.  Used on streams that can be captured and
    // when the profiler is off; a runtime that refuses conditional nodes turns
    // it off for the context (the host-driven loop then runs).
    struct InnerGraph {
        cudaGraphExec_t exec = nullptr;
        const float *gm = nullptr, *r = nullptr;
        float *s = nullptr, *work = nullptr;
        long long N = 0;
        int maxit = 0;
        bool fixed = false;
        double beta0 = 0, gamma = 0;  // baked into the captured transforms
        long k_init = 0, k_head = 0, k_tail = 0;  // kernels of the setup, loop head and tail
    } igr[2];
    double *ictl = nullptr;  // device scalars of the inner solve (16 doubles)
    bool inner_graphs = true;

    // The outer PCG loop of the solver with the InvA preconditioner as one
    // CUDA graph: a conditional WHILE node whose body is one PCG iteration
    // (matvec, update, the device-side stopping test, the preconditioner and
    // the next direction).  Cached per buffer set; the line search alternates
    // the X- buffers, so two variants live at once.
    struct PcgGraph {
        cudaGraphExec_t exec = nullptr;
        const float *dispm = nullptr;
        const int4 *rng = nullptr;
        const float *sv = nullptr;
        int maxit = 0, iorder = 0;
        bool fixed = false;
        double beta = 0, gamma = 0;
        long k_head = 0, k_tail = 0;  // kernels of the loop head and tail
        unsigned long long used = 0;
    } pgr[2];
    unsigned long long pgr_clock = 0;
    double *octl = nullptr;  // device scalars of the outer loop (16 doubles)
    bool pcg_graphs = true;

    void drop_pcg_graphs() {
        for (auto &e : pgr)
            if (e.exec) {
                cudaGraphExecDestroy(e.exec);
                e.exec = nullptr;
            }
    }

    void drop_inner_graphs() {
        for (auto &e : igr)
            if (e.exec) {
                cudaGraphExecDestroy(e.exec);
                e.exec = nullptr;
            }
    }

    // the launches of one inner solve's setup and loop body (captured)
    void inner_setup(const Grid &g, const float *r, float *s, float *work) {
        const long long N = g.d.N, n3 = 3 * N;
        float *ir = work, *iz = ir + n3, *ip = iz + n3, *iAp = ip + n3 + n3;
        const double b0 = beta_h0();
        const SpecParams spb{(float)b0, (float)gamma, (float)(1.0 / (double)N)};
        CK(cudaMemsetAsync(s, 0, n3 * sizeof(float), st));
        CK(cudaMemcpyAsync(ir, r, n3 * sizeof(float), cudaMemcpyDeviceToDevice, st));
        launch_stats(ir, N, partial, ictl + 6, st, &prof);
        launch_inner_init(ictl, st, &prof);
        spectral_apply(g.d, g.ax, OP_AINV, spb, ir, iz, nullptr, g.spec, st, &prof);
        launch_pcg_dir(ip, iAp, iz, ir, ictl + 7, nullptr, 0.f, N, true, st, &prof);
        launch_dot(ir, iz, n3, partial, ictl + 3, st, &prof);
    }
    void inner_head(const Grid &g, const float *gm, float *s, float *work, cudaGraphConditionalHandle h,
                    cudaGraphConditionalHandle h_tail, int maxit, bool fixed) {
        const long long N = g.d.N, n3 = 3 * N;
        float *ir = work, *iz = ir + n3, *ip = iz + n3, *iq = ip + n3, *iAp = iq + n3;
        launch_h0_apply(iq, iAp, gm, ip, N, st, &prof);
        launch_dot(ip, iq, n3, partial, ictl + 2, st, &prof);
        launch_pcg_update(s, nullptr, ir, ip, iAp, iq, 0.f, N, partial, ictl + 6, st, &prof, false, ictl + 2,
                          ictl + 3, nullptr);
        launch_inner_ctl(ictl, h, h_tail, maxit, fixed, st, &prof);
    }
    // the next direction, run only when another iteration follows
    void inner_tail(const Grid &g, float *work) {
        const long long N = g.d.N, n3 = 3 * N;
        float *ir = work, *iz = ir + n3, *ip = iz + n3, *iq = ip + n3, *iAp = iq + n3;
        const double b0 = beta_h0();
        const SpecParams spb{(float)b0, (float)gamma, (float)(1.0 / (double)N)};
        spectral_apply(g.d, g.ax, OP_AINV, spb, ir, iz, nullptr, g.spec, st, &prof);
        launch_dot(ir, iz, n3, partial, ictl + 4, st, &prof);
        launch_pcg_dir(ip, iAp, iz, ir, ictl + 7, nullptr, 0.f, N, false, st, &prof, ictl + 4, ictl + 3);
        launch_scalar_copy(ictl + 3, ictl + 4, st, &prof);
    }

    // builds (or reuses) the graph of grid slot `which` and runs it; false if
    // the runtime refused (nothing has run then)
    bool invh0_graph(const Grid &g, const float *gm, const float *r, float *s, double tol, int maxit, bool fixed,
                     float *work, int which, int &iters) {
        if (!ictl) ictl = (double *)alloc_bytes(16 * sizeof(double));
        InnerGraph &e = igr[which];
        const bool same = e.exec && e.gm == gm && e.r == r && e.s == s && e.work == work && e.N == g.d.N &&
                          e.maxit == maxit && e.fixed == fixed && e.beta0 == beta_h0() && e.gamma == gamma;
        if (!same) {
            if (e.exec) cudaGraphExecDestroy(e.exec);
            e.exec = nullptr;
            const bool ok = build_loop_graph(
                &e.exec, [&] { inner_setup(g, r, s, work); }, true,
                [&](cudaGraphConditionalHandle h, cudaGraphConditionalHandle ht) {
                    inner_head(g, gm, s, work, h, ht, maxit, fixed);
                },
                [&] { inner_tail(g, work); }, e.k_init, e.k_head, e.k_tail);
            if (!ok) {
                inner_graphs = false;
                return false;
            }
            e.gm = gm; e.r = r; e.s = s; e.work = work; e.N = g.d.N; e.maxit = maxit; e.fixed = fixed;
            e.beta0 = beta_h0();
            e.gamma = gamma;
        }
        launch_scalar_set(ictl, tol, st, &prof);
        CK(cudaGraphLaunch(e.exec, st));
        check_launch("invh0 graph");
        double h[11];
        CK(cudaMemcpyAsync(h, ictl, 11 * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        iters = (int)h[5];
        // every loop body runs the head, all but the last one the tail
        prof.launches += e.k_init + (long)h[10] * e.k_head + std::max(0L, (long)h[10] - 1) * e.k_tail;
        return true;
    }

    int invh0_on(const Grid &g, const float *gm, const float *r, float *s, double tol, int maxit,
                 bool fixed, float *work, int which = 0) {
        if (inner_graphs && use_graphs && capturable(st) && !prof.on) {
            int it = 0;
            if (invh0_graph(g, gm, r, s, tol, maxit, fixed, work, which, it)) return it;
        }
        const long long N = g.d.N, n3 = 3 * N;
        float *ir = work, *iz = ir + n3, *ip = iz + n3, *iq = ip + n3, *iAp = iq + n3;
        const double b0 = beta_h0();
        const SpecParams spb{(float)b0, (float)gamma, (float)(1.0 / (double)N)};
        double *slot = dres + 4;
        CK(cudaMemsetAsync(s, 0, n3 * sizeof(float), st));
        CK(cudaMemcpyAsync(ir, r, n3 * sizeof(float), cudaMemcpyDeviceToDevice, st));
        launch_stats(ir, N, partial, slot, st, &prof);
        const double r0 = std::sqrt(fetch(4));
        if (!(r0 > 0)) return 0;
        spectral_apply(g.d, g.ax, OP_AINV, spb, ir, iz, nullptr, g.spec, st, &prof);
        launch_pcg_dir(ip, iAp, iz, ir, slot + 1, nullptr, 0.f, N, true, st, &prof);
        double rz = dot(ir, iz, n3);
        int it = 0;
        while (it < maxit) {
            launch_h0_apply(iq, iAp, gm, ip, N, st, &prof);
            const double pq = dot(ip, iq, n3);
            if (!(pq > 0)) break;
            launch_pcg_update(s, nullptr, ir, ip, iAp, iq, (float)(rz / pq), N, partial, slot, st, &prof);
            ++it;
            const double rn = std::sqrt(fetch(4));
            if (!fixed && rn <= tol * r0) break;
            if (it >= maxit) break;
            spectral_apply(g.d, g.ax, OP_AINV, spb, ir, iz, nullptr, g.spec, st, &prof);
            const double rz_new = dot(ir, iz, n3);
            const float bb = (float)(rz_new / rz);
            rz = rz_new;
            launch_pcg_dir(ip, iAp, iz, ir, slot + 1, nullptr, bb, N, false, st, &prof);
        }
        check_launch("invh0");
        return it;
    }

    // InvH0 (Section 3 "Preconditioning") with grad m(1) of the linearization
    int invh0(const float *r, float *s, double tol, int maxit, bool fixed) {
        if (!have_lin) throw Error(CLAIRE_ERR_STATE, "no linearization (call claire_gradient or claire_linearize)");
        if (!ih) ih = alloc_f((size_t)15 * d.N);
        return invh0_on(fine(), gm_final(), r, s, tol, maxit, fixed, ih);
    }

    // two-level InvH0 (Algorithm 2): restrict r and grad m(1) spectrally to the
    // half grid, solve there, prolong, and add the high-pass part of
    // (beta0 A)^{-1} r -- the last two in one pass over the fine spectrum
    int invh0_2l(const float *r, float *s, double tol, int maxit, bool fixed) {
        if (!have_lin) throw Error(CLAIRE_ERR_STATE, "no linearization (call claire_gradient or claire_linearize)");
        make_coarse();
        const Grid cg{co.d, co.ax, co.spec};
        const float c2f = (float)((double)d.N / (double)co.d.N), f2c = 1.f / c2f;
        if (!co.gm_valid) {
            spectral_forward3(d, ax, gm_final(), spec, st, &prof);
            launch_spec_restrict(d, spec, co.d, co.spec, f2c, st, &prof);
            spectral_inverse3(co.d, co.ax, co.spec, co.gm, (float)(1.0 / (double)co.d.N), st, &prof);
            co.gm_valid = true;
        }
        spectral_forward3(d, ax, r, spec, st, &prof);
        launch_spec_restrict(d, spec, co.d, co.spec, f2c, st, &prof);
        spectral_inverse3(co.d, co.ax, co.spec, co.r, (float)(1.0 / (double)co.d.N), st, &prof);
        const int it = invh0_on(cg, co.gm, co.r, co.s, tol, maxit, fixed, co.work, 1);
        spectral_forward3(co.d, co.ax, co.s, co.spec, st, &prof);
        launch_spec_twolevel(d, spec, co.d, co.spec, c2f, (float)beta_h0(), (float)gamma, st, &prof);
        spectral_inverse3(d, ax, spec, s, (float)(1.0 / (double)d.N), st, &prof);
        check_launch("invh0_2l");
        return it;
    }

    // first derivatives by the selected discretization
    void grad(const float *f, float *g) {
        if (deriv_fd8) launch_grad_fd8(d, f, g, st, &prof);
        else spectral_grad_1d(d, ax, f, g, st, &prof);
    }
    void grad_h(const float *f, __half *g) {
        if (deriv_fd8) launch_grad_fd8(d, f, g, st, &prof);
        else spectral_grad_1d(d, ax, f, g, st, &prof);
    }
    void div(const float *v, float *out) { div_on(v, out, st); }
    void div_on(const float *v, float *out, cudaStream_t s) {
        if (deriv_fd8) launch_div_fd8(d, v, out, s, &prof);
        else spectral_div_1d(d, ax, v, out, s, &prof);
    }

    // a second stream for work that runs beside the main one (created on
    // first use, with its fork and join events)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    void ensure_side() {
        if (side) return;
        // all three or none: a failure leaves the context as it was
        cudaStream_t s = nullptr;
        cudaEvent_t f = nullptr, j = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            if (j) cudaEventDestroy(j);
            if (f) cudaEventDestroy(f);
            if (s) cudaStreamDestroy(s);
            CK(e);
        }
        side = s;
        ev_fork = f;
        ev_join = j;
    }

    // With state_ready, mhist and dispm already hold the state and the X- foot
    // points of v (an adopted line-search trial); only X+ is computed here.
    void linearize(const float *v, bool state_ready = false) {
        if (!have_images) throw Error(CLAIRE_ERR_STATE, "images not set (claire_set_images)");
        const size_t N = d.N;
        if (v != vlin) CK(cudaMemcpyAsync(vlin, v, 3 * N * sizeof(float), cudaMemcpyDeviceToDevice, st));
        // After an adopted trial only X+, div v and c remain besides grad m^j,
        // and they do not depend on it: they run on a second stream while the
        // gradients run on the context's (joined before returning).  Not while
        // the profiler times launches one by one.
        const bool fork = state_ready && !h16 && !prof.on;
        if (fork) {
            ensure_side();
            CK(cudaEventRecord(ev_fork, st));
            CK(cudaStreamWaitEvent(side, ev_fork, 0));
            launch_footpoints(d, nt, vlin, nullptr, dispp, nullptr, rng_p(), side, &prof);
            div_on(vlin, divv, side);
            launch_adjoint_factor(d, nt, divv, dispp, rng_p(), cfac, side, &prof);
            CK(cudaEventRecord(ev_join, side));
            for (int j = gm0_valid ? 1 : 0; j <= nt; ++j) grad(hist(mhist, j), hist(gmhist, j, 3));
            gm0_valid = true;
            CK(cudaStreamWaitEvent(st, ev_join, 0));
            check_launch("linearize");
            ++lin_epoch;
            have_lin = true;
            co.gm_valid = false;
            return;
        }
        if (state_ready) {
            launch_footpoints(d, nt, vlin, nullptr, dispp, nullptr, rng_p(), st, &prof);
        } else if (h16) {
            // FP32 transport; FP16 copies of m^j and of grad m^j (taken of the
            // FP32 state); m(1) and grad m(1) also kept in FP32
            launch_footpoints(d, nt, vlin, dispm, dispp, rng_m(), rng_p(), st, &prof);
            wait_images();
            launch_f2h(m0, mhist_h, (long long)N, st, &prof);
            if (!gm0_valid) grad_h(m0, hist(gmhist_h, 0, 3));
            const float *src = m0;
            float *a = s1a, *b = s1b;
            for (int j = 0; j < nt; ++j) {
                float *dst = j + 1 == nt ? m1f : a;
                launch_state_step(d, src, dispm, rng_m(), dst, st, &prof, hist(mhist_h, j + 1));
                if (j + 1 < nt) grad_h(dst, hist(gmhist_h, j + 1, 3));
                src = dst;
                std::swap(a, b);
            }
            grad(m1f, gm1f);
            launch_f2h(gm1f, hist(gmhist_h, nt, 3), 3 * (long long)N, st, &prof);
        } else if (!prof.on) {
            // X+, div v and c on the second stream while X-, the state and
            // grad m^j run on the context's (the same kernels as below, side
            // by side; joined before returning)
            ensure_side();
            CK(cudaEventRecord(ev_fork, st));
            CK(cudaStreamWaitEvent(side, ev_fork, 0));
            launch_footpoints(d, nt, vlin, nullptr, dispp, nullptr, rng_p(), side, &prof);
            div_on(vlin, divv, side);
            launch_adjoint_factor(d, nt, divv, dispp, rng_p(), cfac, side, &prof);
            CK(cudaEventRecord(ev_join, side));
            launch_footpoints(d, nt, vlin, dispm, nullptr, rng_m(), nullptr, st, &prof);
            wait_images();
            CK(cudaMemcpyAsync(mhist, m0, N * sizeof(float), cudaMemcpyDeviceToDevice, st));
            for (int j = 0; j < nt; ++j)
                launch_state_step(d, hist(mhist, j), dispm, rng_m(), hist(mhist, j + 1), st, &prof);
            for (int j = gm0_valid ? 1 : 0; j <= nt; ++j) grad(hist(mhist, j), hist(gmhist, j, 3));
            gm0_valid = true;
            CK(cudaStreamWaitEvent(st, ev_join, 0));
            check_launch("linearize");
            ++lin_epoch;
            have_lin = true;
            co.gm_valid = false;
            return;
        } else {
            launch_footpoints(d, nt, vlin, dispm, dispp, rng_m(), rng_p(), st, &prof);
            wait_images();
            CK(cudaMemcpyAsync(mhist, m0, N * sizeof(float), cudaMemcpyDeviceToDevice, st));
            for (int j = 0; j < nt; ++j)
                launch_state_step(d, hist(mhist, j), dispm, rng_m(), hist(mhist, j + 1), st, &prof);
        }
        wait_images();
        if (!h16)
            for (int j = gm0_valid ? 1 : 0; j <= nt; ++j) grad(hist(mhist, j), hist(gmhist, j, 3));
        gm0_valid = true;
        div(vlin, divv);
        launch_adjoint_factor(d, nt, divv, dispp, rng_p(), cfac, st, &prof);
        check_launch("linearize");
        ++lin_epoch;
        have_lin = true;
        co.gm_valid = false;
    }

    // adjoint solve + body force + beta A v; J into *J when asked.  Av, if
    // given, is beta*A v already at hand (the solver carries it along);
    // otherwise it is applied spectrally.
    void gradient(const float *v, float *g, double *J, double *mis_out, const float *Av = nullptr,
                  bool state_ready = false) {
        linearize(v, state_ready);
        const size_t N = d.N;
        if (!Av) {
            spectral(OP_A, vlin, s3a, nullptr);
            Av = s3a;
        }
        // g = beta A v + the body force of Eq. 3.3 by the trapezoidal rule,
        // each term added by the adjoint step that makes its lambda^j; the
        // last step also leaves g . g in dres[9]
        const float dt = 1.f / nt;
        auto wt = [&](int j) { return (j == 0 || j == nt) ? 0.5f * dt : dt; };
        if (h16) {
            // FP32 adjoint transport with FP16 copies of lambda^j
            float *a = s1a, *b = s1b;
            launch_adjfinal_acc(d, m1, m1f, a, hist(lhist_h, nt), hist(gmhist_h, nt, 3), Av, g, wt(nt), st, &prof);
            for (int j = nt; j >= 1; --j) {
                launch_adjoint_acc(d, a, dispp, rng_p(), cfac, b, hist(gmhist_h, j - 1, 3), g, wt(j - 1), j == 1,
                                   nullptr, partial, nullptr, dres + 9, st, &prof, CLAIRE_K_ADJOINT,
                                   hist(lhist_h, j - 1));
                std::swap(a, b);
            }
        } else {
            launch_adjfinal_acc(d, m1, hist(mhist, nt), hist(lhist, nt), nullptr, hist(gmhist, nt, 3), Av, g, wt(nt),
                                st, &prof);
            for (int j = nt; j >= 1; --j)
                launch_adjoint_acc(d, hist(lhist, j), dispp, rng_p(), cfac, hist(lhist, j - 1), hist(gmhist, j - 1, 3),
                                   g, wt(j - 1), j == 1, nullptr, partial, nullptr, dres + 9, st, &prof,
                                   CLAIRE_K_ADJOINT);
        }
        check_launch("gradient");
        if (J || mis_out) {
            const double H3 = h3();
            const double mis = h16 ? final_mismatch() : 0.5 * H3 * dot(hist(lhist, nt), hist(lhist, nt), (long long)N);
            last_vAv = dot(vlin, Av, 3 * (long long)N);
            const double reg = 0.5 * H3 * last_vAv;
            if (J) *J = mis + reg;
            if (mis_out) *mis_out = mis;
        }
    }

    // CUDA graph of the matvec's launch sequence.  The PCG loop calls the
    // matvec with the same buffers every iteration of a linearization, so the
    // second call with a given signature is captured and later ones replay
    // the graph (one launch instead of ~12).  Off on the legacy stream (no
    // capture there) and while the profiler records per-launch events.
    struct MvGraph {
        cudaGraphExec_t exec = nullptr;
        const float *vt = nullptr;
        float *Hvt = nullptr;
        unsigned long long epoch = ~0ULL;
        int seen = 0;       // calls with this signature so far
        long kernels = 0;   // kernel launches one replay stands for
        bool same(const float *a, float *b, unsigned long long e) const {
            return vt == a && Hvt == b && epoch == e;
        }
    } mvg;
    unsigned long long lin_epoch = 0;  // bumped by every linearization
    bool use_graphs = true;

    // Hvt = beta A vt + int lt grad m dt (Eq. 3.4-3.6).  The PCG form (pcg):
    // s1a already holds u0 = dt/2 f^0 and dres[8] holds vt . beta A vt (both
    // written by the PCG direction update, launch_pcg_dir_u0); Hvt receives
    // the body force only (the PCG update adds beta A vt, which it carries)
    // and dres[0] receives vt . H vt.
    void matvec(const float *vt, float *Hvt, bool pcg = false) {
        if (!have_lin) throw Error(CLAIRE_ERR_STATE, "no linearization (call claire_gradient or claire_linearize)");
        const bool graph = use_graphs && pcg && capturable(st) && !prof.on;
        if (graph) {
            if (mvg.same(vt, Hvt, lin_epoch)) {
                if (mvg.exec) {
                    CK(cudaGraphLaunch(mvg.exec, st));
                    prof.launches += mvg.kernels;
                    return;
                }
                if (mvg.seen >= 1 && capture_matvec(vt, Hvt)) return;
            } else {
                drop_graph();
                mvg.vt = vt; mvg.Hvt = Hvt;
                mvg.epoch = lin_epoch;
                mvg.seen = 0;
            }
            ++mvg.seen;
        }
        matvec_launches(vt, Hvt, pcg);
        check_launch("hess_matvec");
    }

    void drop_graph() {
        if (mvg.exec) cudaGraphExecDestroy(mvg.exec);
        mvg.exec = nullptr;
    }

    // streams a graph can be captured on (not the legacy or per-thread
    // default streams)
    static bool capturable(cudaStream_t s) {
        return s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread;
    }

    // captures and runs the matvec as a graph; false (and graphs off for this
    // context, the launches not yet run) if the runtime refuses the capture
    bool capture_matvec(const float *vt, float *Hvt) {
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            use_graphs = false;
            return false;
        }
        const long before = prof.launches;
        try {
            matvec_launches(vt, Hvt, true);
            mvg.kernels = prof.launches - before;
        } catch (...) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(st, &g);
            if (g) cudaGraphDestroy(g);
            throw;
        }
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(st, &g);
        if (e == cudaSuccess && g) e = cudaGraphInstantiate(&mvg.exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess || !mvg.exec) {
            cudaGetLastError();
            mvg.exec = nullptr;
            prof.launches = before;
            use_graphs = false;
            return false;
        }
        CK(cudaGraphLaunch(mvg.exec, st));
        check_launch("hess_matvec graph");
        return true;
    }

    void matvec_launches(const float *vt, float *Hvt, bool pcg) {
        const float dt = 1.f / nt;
        float *u = s1a, *un = s1b;
        if (!pcg) {
            if (h16) launch_incstate_init(d, dt, vt, hist(gmhist_h, 0, 3), u, st, &prof);
            else launch_incstate_init(d, dt, vt, hist(gmhist, 0, 3), u, st, &prof);
        }
        for (int j = 0; j + 1 < nt; ++j) {
            if (h16) launch_incstate_step(d, dt, u, dispm, rng_m(), vt, hist(gmhist_h, j + 1, 3), un, st, &prof);
            else launch_incstate_step(d, dt, u, dispm, rng_m(), vt, hist(gmhist, j + 1, 3), un, st, &prof);
            float *t = u; u = un; un = t;
        }
        // the last step writes the incremental adjoint's final condition and
        // starts the body force (Eq. 3.6) in Hvt; every incremental-adjoint
        // step adds its own trapezoid term, the last one also forms vt . H vt
        if (h16)
            launch_incstate_last(d, dt, u, dispm, rng_m(), vt, hist(gmhist_h, nt, 3), hist(lhist, nt), mt, Hvt, st,
                                 &prof);
        else
            launch_incstate_last(d, dt, u, dispm, rng_m(), vt, hist(gmhist, nt, 3), hist(lhist, nt), mt, Hvt, st,
                                 &prof);
        for (int j = nt; j >= 1; --j) {
            const float w = j == 1 ? 0.5f * dt : dt;
            const bool dot = pcg && j == 1;
            if (h16)
                launch_adjoint_acc(d, hist(lhist, j), dispp, rng_p(), cfac, hist(lhist, j - 1), hist(gmhist_h, j - 1, 3),
                                   Hvt, w, dot, vt, partial, dres + 8, dres, st, &prof, CLAIRE_K_INCADJ);
            else
                launch_adjoint_acc(d, hist(lhist, j), dispp, rng_p(), cfac, hist(lhist, j - 1), hist(gmhist, j - 1, 3),
                                   Hvt, w, dot, vt, partial, dres + 8, dres, st, &prof, CLAIRE_K_INCADJ);
        }
        if (!pcg) spectral(OP_A, vt, Hvt, Hvt);
    }

    // ---- differentiable transport with state checkpointing -----------------
    // checkpoints m^j at j = 0, k, 2k, ... and nt; a buffer for the states of
    // one segment (recomputed in the backward pass; none when k = 1, where
    // every state is a checkpoint); one gradient buffer (each grad m^j is
    // taken once, right before its body-force term)
    float *ck = nullptr, *seg_m = nullptr, *gbuf = nullptr, *bacc = nullptr, *lam2 = nullptr;
    int ck_stride = 0;
    bool ck_valid = false;
    int n_ck() const { return (nt + ck_stride - 1) / ck_stride + 1; }
    int ck_slot(int j) const { return j == nt ? n_ck() - 1 : j / ck_stride; }
    // floats of N the differentiable form holds for stride k
    long long ck_fields(int k) const { return (nt + k - 1) / k + 1 + (k > 1 ? k + 1 : 0) + 3 + 3 + 2; }

    // stride for checkpoint_stride = 0: keep every state (no recomputation)
    // when that fits the memory left (the device's free memory less a reserve,
    // and the workspace cap if one is set); otherwise the stride that needs
    // the least memory; CLAIRE_ERR_OOM if even that does not fit
    int auto_stride() const {
        size_t free_b = 0, total_b = 0;
        CK(cudaMemGetInfo(&free_b, &total_b));
        const size_t reserve = 256ull << 20;
        double budget = free_b > reserve ? (double)(free_b - reserve) : 0.0;
        const size_t cap = g_workspace_limit.load();
        if (cap) budget = std::min(budget, cap > bytes ? (double)(cap - bytes) : 0.0);
        const double fb = 4.0 * (double)d.N;
        if ((double)ck_fields(1) * fb <= budget) return 1;
        int best = 1;
        for (int k = 2; k <= nt; ++k)
            if (ck_fields(k) < ck_fields(best)) best = k;
        if ((double)ck_fields(best) * fb > budget)
            throw Error(CLAIRE_ERR_OOM, "differentiable form: no checkpoint stride fits the free device memory");
        return best;
    }

    void ensure_ck(int stride) {
        if (stride != ck_stride) {
            if (ck) throw Error(CLAIRE_ERR_STATE, "checkpoint stride is fixed after the first differentiable forward");
            // all or nothing: a failed allocation leaves the context as it was
            const size_t mark = allocs.size(), bytes0 = bytes;
            try {
                float *c0 = alloc_f((size_t)((nt + stride - 1) / stride + 1) * d.N);
                float *c1 = stride > 1 ? alloc_f((size_t)(stride + 1) * d.N) : nullptr;
                float *c2 = alloc_f(3 * (size_t)d.N);
                float *c3 = alloc_f(3 * (size_t)d.N);
                float *c4 = alloc_f(2 * (size_t)d.N);
                ck = c0;
                seg_m = c1;
                gbuf = c2;
                bacc = c3;
                lam2 = c4;
                ck_stride = stride;
            } catch (...) {
                rollback(mark, bytes0);
                throw;
            }
        }
    }

    // forward transport keeping only checkpoints; X-, X+ and c at v kept for
    // the backward; returns the mismatch 1/2 ||m(1) - m1||^2.  stride 0: the
    // stride is chosen from the free memory (auto_stride) at the first call
    double diff_forward(const float *v, float *m_final, int stride) {
        if (!have_images) throw Error(CLAIRE_ERR_STATE, "images not set (claire_set_images)");
        if (stride == 0) stride = ck_stride ? ck_stride : auto_stride();
        ensure_ck(stride);
        const size_t N = d.N;
        if (v != vlin) CK(cudaMemcpyAsync(vlin, v, 3 * N * sizeof(float), cudaMemcpyDeviceToDevice, st));
        have_lin = false;  // the full history is not kept on this path
        launch_footpoints(d, nt, vlin, dispm, dispp, rng_m(), rng_p(), st, &prof);
        div(vlin, divv);
        launch_adjoint_factor(d, nt, divv, dispp, rng_p(), cfac, st, &prof);
        CK(cudaMemcpyAsync(ck, m0, N * sizeof(float), cudaMemcpyDeviceToDevice, st));
        const float *src = m0;
        float *a = s1a, *b = s1b;
        for (int j = 0; j < nt; ++j) {
            const int jn = j + 1;
            float *dst = (jn % ck_stride == 0 || jn == nt) ? ck + (size_t)ck_slot(jn) * N : a;
            launch_state_step(d, src, dispm, rng_m(), dst, st, &prof);
            src = dst;
            if (dst == a) { float *t = a; a = b; b = t; }
        }
        ck_valid = true;
        const float *mT = ck + (size_t)ck_slot(nt) * N;
        if (m_final) CK(cudaMemcpyAsync(m_final, mT, N * sizeof(float), cudaMemcpyDeviceToDevice, st));
        check_launch("mismatch_forward");
        return mismatch_of(mT);
    }

    // backward of (mismatch, m(1)) -> v: adjoint from l(1) = gmis (m1 - m(1))
    // - gm_final / h^3, segments recomputed from the checkpoints (none when
    // every state is a checkpoint), body force accumulated by the trapezoidal
    // rule level by level from t = 1 down to 0, each grad m^j taken once;
    // grad_v = h^3 b (Euclidean)
    void diff_backward(double gmis, const float *gm_final, float *grad_v) {
        if (!ck_valid) throw Error(CLAIRE_ERR_STATE, "no differentiable forward at this point");
        const size_t N = d.N;
        const double H3 = h3();
        const float dt = 1.f / nt;
        float *lam = lam2, *lam_next = lam2 + N;
        launch_adjoint_final(d, lam, m1, ck + (size_t)ck_slot(nt) * N, gm_final, (float)gmis,
                             (float)(1.0 / H3), st, &prof);
        CK(cudaMemsetAsync(bacc, 0, 3 * N * sizeof(float), st));
        const int nseg = (nt + ck_stride - 1) / ck_stride;
        for (int sgi = nseg - 1; sgi >= 0; --sgi) {
            const int j0 = sgi * ck_stride, j1 = std::min(j0 + ck_stride, nt);
            // the states m^j, j0..j1, of the segment: the checkpoints
            // themselves for stride 1, else recomputed from m^{j0}
            auto state = [&](int j) -> const float * {
                if (ck_stride == 1) return ck + (size_t)ck_slot(j) * N;
                return seg_m + (size_t)(j - j0) * N;
            };
            if (ck_stride > 1) {
                CK(cudaMemcpyAsync(seg_m, ck + (size_t)ck_slot(j0) * N, N * sizeof(float), cudaMemcpyDeviceToDevice,
                                   st));
                for (int j = j0; j < j1; ++j)
                    launch_state_step(d, seg_m + (size_t)(j - j0) * N, dispm, rng_m(), seg_m + (size_t)(j + 1 - j0) * N,
                                      st, &prof);
            }
            // body-force terms of levels j1 .. j0+1 with the adjoint steps
            // j1 -> j0 (and the level j0 = 0 term at the very end)
            for (int j = j1; j > j0; --j) {
                const float w = (j == nt ? 0.5f : 1.f) * dt;
                grad(state(j), gbuf);
                launch_bodyforce_acc(d, bacc, lam, gbuf, w, st, &prof);
                launch_adjoint_step(d, lam, dispp, rng_p(), cfac, lam_next, st, &prof, CLAIRE_K_ADJOINT);
                float *t = lam; lam = lam_next; lam_next = t;
            }
            if (j0 == 0) {
                grad(state(0), gbuf);
                launch_bodyforce_acc(d, bacc, lam, gbuf, 0.5f * dt, st, &prof);
            }
        }
        launch_axpby(grad_v, (float)H3, bacc, 0.f, nullptr, 3 * (long long)N, st, &prof);
        check_launch("mismatch_backward");
    }

    // m(1) for v into mout (N); uses fdisp, s1a, s1b; leaves the cache alone
    const float *forward(const float *v) {
        if (!have_images) throw Error(CLAIRE_ERR_STATE, "images not set (claire_set_images)");
        launch_footpoints(d, nt, v, fdisp, nullptr, rng_f(), nullptr, st, &prof);
        const float *src = m0;
        float *a = s1a, *b = s1b;
        for (int j = 0; j < nt; ++j) {
            launch_state_step(d, src, fdisp, rng_f(), a, st, &prof);
            src = a;
            float *t = a; a = b; b = t;
        }
        check_launch("forward");
        return src;
    }

    // the forward solve of the line search; returns 1/2 h^3 ||m(1) - m1||^2.
    // The FP32 form keeps the trial's states (m^j into mhist_t, X- in fdisp):
    // an accepted trial becomes the next linearization as it stands.  The
    // FP16-storage form stores grad m^j of the FP32 states, which the trial does
    // not make, so it transports in FP32 scratch and its linearization
    // recomputes the state.
    bool keeps_trial() const { return !h16; }
    double trial_mismatch(const float *v) {
        if (h16) return mismatch_of(forward(v));
        launch_footpoints(d, nt, v, fdisp, nullptr, rng_f(), nullptr, st, &prof);
        if (!mhist_t) mhist_t = alloc_f((size_t)(nt + 1) * d.N);
        const float *src = m0;
        for (int j = 0; j < nt; ++j) {
            launch_state_step(d, src, fdisp, rng_f(), hist(mhist_t, j + 1), st, &prof);
            src = hist(mhist_t, j + 1);
        }
        check_launch("forward_trial");
        return mismatch_of(src);
    }
    // the last trial's state and foot points become those of the linearization
    void adopt_trial() {
        std::swap(dispm, fdisp);
        std::swap(off_m, off_f);
        std::swap(mhist, mhist_t);
        CK(cudaMemcpyAsync(mhist, m0, d.N * sizeof(float), cudaMemcpyDeviceToDevice, st));
    }
    // 1/2 h^3 ||m(1) - m1||^2 of the linearization's state
    double final_mismatch() {
        launch_sqdiff(h16 ? m1f : hist(mhist, nt), m1, d.N, partial, dres, st, &prof);
        return 0.5 * h3() * fetch();
    }

    double mismatch_of(const float *mfinal) {
        launch_sqdiff(mfinal, m1, d.N, partial, dres, st, &prof);
        return 0.5 * h3() * fetch();
    }

    double objective(const float *v, double *mis_out) {
        const float *mf = forward(v);
        const double mis = mismatch_of(mf);
        spectral(OP_A, v, s3a, nullptr);
        const double reg = 0.5 * h3() * dot(v, s3a, 3 * d.N);
        if (mis_out) *mis_out = mis;
        return mis + reg;
    }
};

// -------------------------------------------------------------- helpers ----
// NVTX range for an external profiler's timeline (named after the ABI call
// or the solver phase); costs a few host instructions when no tool listens
struct Nvtx {
    explicit Nvtx(const char *name) { nvtxRangePushA(name); }
    ~Nvtx() { nvtxRangePop(); }
    Nvtx(const Nvtx &) = delete;
    Nvtx &operator=(const Nvtx &) = delete;
};

#define API_BEGIN(ctx)                                                        \
    if (!(ctx)) return CLAIRE_ERR_ARG;                                        \
    Nvtx nvtx_call_(__func__);                                                \
    try {
#define API_END(ctx)                                                          \
    }                                                                         \
    catch (const Error &e) {                                                  \
        (ctx)->err = e.msg;                                                   \
        return e.code;                                                        \
    }                                                                         \
    catch (const std::bad_alloc &) {                                          \
        (ctx)->err = "host allocation failed";                                \
        return CLAIRE_ERR_OOM;                                                \
    }                                                                         \
    catch (const std::exception &e) {                                         \
        (ctx)->err = e.what();                                                \
        return CLAIRE_ERR_CUDA;                                               \
    }                                                                         \
    return CLAIRE_OK;

static void need(const void *p, const char *name) {
    if (!p) throw Error(CLAIRE_ERR_ARG, std::string(name) + " is NULL");
}

static void check_params(double beta, double gamma) {
    if (!(beta > 0) || !std::isfinite(beta)) throw Error(CLAIRE_ERR_ARG, "beta must be finite and > 0");
    if (!(gamma >= 0) || !std::isfinite(gamma)) throw Error(CLAIRE_ERR_ARG, "gamma must be finite and >= 0");
}

// ------------------------------------------------------------------- ABI ---
extern "C" {

int claire_create(int nx, int ny, int nz, int nt, double beta, double gamma, claire_ctx **out) {
    return claire_create_ex(nx, ny, nz, nt, beta, gamma, CLAIRE_PREC_FP32, out);
}

int claire_create_ex(int nx, int ny, int nz, int nt, double beta, double gamma, int precision,
                     claire_ctx **out) {
    if (!out) {
        g_create_error = "out is NULL";
        return CLAIRE_ERR_ARG;
    }
    *out = nullptr;
    if (!valid_n(nx) || !valid_n(ny) || !valid_n(nz)) {
        g_create_error = "grid sizes must be in [4, 1024] with prime factors 2, 3, 5 only";
        return CLAIRE_ERR_ARG;
    }
    if (nt < 1 || nt > 256) {
        g_create_error = "nt must be in [1, 256]";
        return CLAIRE_ERR_ARG;
    }
    if (precision != CLAIRE_PREC_FP32 && precision != CLAIRE_PREC_FP16_STORAGE) {
        g_create_error = "unknown precision mode";
        return CLAIRE_ERR_ARG;
    }
    claire_ctx *c = nullptr;
    try {
        check_params(beta, gamma);
        c = new claire_ctx();
        c->h16 = precision == CLAIRE_PREC_FP16_STORAGE;
        c->d.n1 = nx;
        c->d.n2 = ny;
        c->d.n3 = nz;
        c->d.N = (long long)nx * ny * nz;
        c->d.h3 = nz / 2 + 1;
        c->d.p3 = (c->d.h3 + 3) / 4 * 4;
        c->nt = nt;
        c->beta = beta;
        c->gamma = gamma;
        const int ns[3] = {nx, ny, nz};
        for (int a = 0; a < 3; ++a) {
            c->ax[a] = make_plan(ns[a]);
            std::vector<float2> tw(ns[a]);
            for (int t = 0; t < ns[a]; ++t) {
                const double ang = 6.283185307179586476925286766559 * (double)t / (double)ns[a];
                tw[t] = make_float2((float)std::cos(ang), (float)(-std::sin(ang)));
            }
            float2 *dtw = nullptr;
            CK(cudaMalloc(&dtw, ns[a] * sizeof(float2)));
            c->ax[a].tw = dtw;
            CK(cudaMemcpy(dtw, tw.data(), ns[a] * sizeof(float2), cudaMemcpyHostToDevice));
        }
        const size_t N = c->d.N;
        c->m0 = c->alloc_f(N);
        c->m1 = c->alloc_f(N);
        c->vlin = c->alloc_f(3 * N);
        c->dispm = c->alloc_f(3 * N);
        c->dispp = c->alloc_f(3 * N);
        if (c->h16) {
            c->mhist_h = c->alloc_h((size_t)(nt + 1) * N);
            c->gmhist_h = c->alloc_h((size_t)(nt + 1) * 3 * N);
            c->lhist_h = c->alloc_h((size_t)(nt + 1) * N);
            c->gm1f = c->alloc_f(3 * N);
            c->m1f = c->alloc_f(N);
        } else {
            c->mhist = c->alloc_f((size_t)(nt + 1) * N);
            c->gmhist = c->alloc_f((size_t)(nt + 1) * 3 * N);
        }
        c->divv = c->alloc_f(N);
        c->cfac = c->alloc_f(N);
        c->lhist = c->alloc_f((size_t)(nt + 1) * N);
        c->mt = c->alloc_f(N);
        c->s3a = c->alloc_f(3 * N);
        c->s1a = c->alloc_f(N);
        c->s1b = c->alloc_f(N);
        c->fdisp = c->alloc_f(3 * N);
        c->spec = (float2 *)c->alloc_bytes((size_t)3 * nx * ny * c->d.p3 * sizeof(float2));
        c->partial = (double *)c->alloc_bytes(4 * kReduceBlocks * sizeof(double));
        c->dres = (double *)c->alloc_bytes(16 * sizeof(double));
        c->dflag = (int *)c->alloc_bytes(sizeof(int));
        c->ntiles = tile_count(c->d);
        c->rng = (int4 *)c->alloc_bytes((size_t)4 * c->ntiles * sizeof(int4));
    } catch (const Error &e) {
        g_create_error = e.msg;
        delete c;
        return e.code;
    } catch (const std::bad_alloc &) {
        g_create_error = "host allocation failed";
        delete c;
        return CLAIRE_ERR_OOM;
    }
    *out = c;
    return CLAIRE_OK;
}

int claire_destroy(claire_ctx *ctx) {
    if (!ctx) return CLAIRE_OK;
    cudaStreamSynchronize(ctx->st);
    delete ctx;
    return CLAIRE_OK;
}

int claire_set_stream(claire_ctx *ctx, void *stream) {
    API_BEGIN(ctx)
    ctx->st = (cudaStream_t)stream;
    API_END(ctx)
}

int claire_set_params(claire_ctx *ctx, double beta, double gamma) {
    API_BEGIN(ctx)
    check_params(beta, gamma);
    ctx->beta = beta;
    ctx->gamma = gamma;
    API_END(ctx)
}

int claire_set_images(claire_ctx *ctx, const float *m0, const float *m1) {
    API_BEGIN(ctx)
    need(m0, "m0");
    need(m1, "m1");
    const size_t b = ctx->d.N * sizeof(float);
    CK(cudaMemcpyAsync(ctx->m0, m0, b, cudaMemcpyDeviceToDevice, ctx->st));
    CK(cudaMemcpyAsync(ctx->m1, m1, b, cudaMemcpyDeviceToDevice, ctx->st));
    ctx->have_images = true;
    ctx->have_lin = false;
    ctx->gm0_valid = false;
    API_END(ctx)
}

int claire_forward(claire_ctx *ctx, const float *v, float *m_final, double *mismatch) {
    API_BEGIN(ctx)
    need(v, "v");
    const float *mf = ctx->forward(v);
    if (m_final)
        CK(cudaMemcpyAsync(m_final, mf, ctx->d.N * sizeof(float), cudaMemcpyDeviceToDevice, ctx->st));
    if (mismatch) *mismatch = ctx->mismatch_of(mf);
    API_END(ctx)
}

int claire_objective(claire_ctx *ctx, const float *v, double *objective, double *mismatch) {
    API_BEGIN(ctx)
    need(v, "v");
    need(objective, "objective");
    *objective = ctx->objective(v, mismatch);
    API_END(ctx)
}

int claire_linearize(claire_ctx *ctx, const float *v) {
    API_BEGIN(ctx)
    need(v, "v");
    ctx->linearize(v);
    API_END(ctx)
}

int claire_gradient(claire_ctx *ctx, const float *v, float *g, double *objective) {
    API_BEGIN(ctx)
    need(v, "v");
    need(g, "g");
    ctx->gradient(v, g, objective, nullptr);
    API_END(ctx)
}

int claire_hess_matvec(claire_ctx *ctx, const float *v, const float *vt, float *Hvt) {
    API_BEGIN(ctx)
    need(vt, "vt");
    need(Hvt, "Hvt");
    if (vt == Hvt) throw Error(CLAIRE_ERR_ARG, "vt and Hvt may not alias");
    if (v) {
        bool same = false;
        if (ctx->have_lin) {
            launch_diff_flag(v, ctx->vlin, 3 * ctx->d.N, ctx->dflag, ctx->st, &ctx->prof);
            int h = 1;
            CK(cudaMemcpyAsync(&h, ctx->dflag, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
            CK(cudaStreamSynchronize(ctx->st));
            same = (h == 0);
        }
        if (!same) ctx->linearize(v);
    }
    ctx->matvec(vt, Hvt);
    API_END(ctx)
}

int claire_precond(claire_ctx *ctx, const float *r, float *s) {
    API_BEGIN(ctx)
    need(r, "r");
    need(s, "s");
    ctx->spectral(OP_AINV, r, s, nullptr);
    check_launch("precond");
    API_END(ctx)
}

int claire_mismatch_forward(claire_ctx *ctx, const float *v, float *m_final, double *mismatch,
                            int checkpoint_stride) {
    API_BEGIN(ctx)
    need(v, "v");
    if (checkpoint_stride < 0 || checkpoint_stride > ctx->nt)
        throw Error(CLAIRE_ERR_ARG, "checkpoint_stride must be in [0, nt] (0: chosen from the free memory)");
    const double mis = ctx->diff_forward(v, m_final, checkpoint_stride);
    if (mismatch) *mismatch = mis;
    API_END(ctx)
}

int claire_checkpoint_stride(const claire_ctx *ctx, int *stride) {
    if (!ctx || !stride) return CLAIRE_ERR_ARG;
    *stride = ctx->ck_stride;
    return CLAIRE_OK;
}
int claire_mismatch_backward(claire_ctx *ctx, double grad_mismatch, const float *grad_m_final,
                             float *grad_v) {
    API_BEGIN(ctx)
    need(grad_v, "grad_v");
    if (!std::isfinite(grad_mismatch)) throw Error(CLAIRE_ERR_NONFINITE, "non-finite upstream gradient");
    ctx->diff_backward(grad_mismatch, grad_m_final, grad_v);
    API_END(ctx)
}

int claire_precond_h0(claire_ctx *ctx, const float *r, float *s, double tol, int maxit,
                      int two_level, int *iterations) {
    API_BEGIN(ctx)
    need(r, "r");
    need(s, "s");
    if (r == s) throw Error(CLAIRE_ERR_ARG, "r and s may not alias");
    if (maxit < 1 || !(tol >= 0)) throw Error(CLAIRE_ERR_ARG, "need maxit >= 1 and tol >= 0");
    const int it = two_level ? ctx->invh0_2l(r, s, tol, maxit, tol == 0.0)
                             : ctx->invh0(r, s, tol, maxit, tol == 0.0);
    if (iterations) *iterations = it;
    API_END(ctx)
}

int claire_set_discretization(claire_ctx *ctx, int interp_order, int deriv) {
    API_BEGIN(ctx)
    if (interp_order != 1 && interp_order != 3) throw Error(CLAIRE_ERR_ARG, "interp_order must be 1 or 3");
    if (deriv != CLAIRE_DERIV_SPECTRAL && deriv != CLAIRE_DERIV_FD8) throw Error(CLAIRE_ERR_ARG, "unknown derivative scheme");
    ctx->d.iorder = interp_order;
    ctx->deriv_fd8 = deriv == CLAIRE_DERIV_FD8;
    ctx->have_lin = false;
    ctx->gm0_valid = false;
    API_END(ctx)
}

int claire_grad(claire_ctx *ctx, const float *f, float *g) {
    API_BEGIN(ctx)
    need(f, "f");
    need(g, "g");
    ctx->grad(f, g);
    check_launch("grad");
    API_END(ctx)
}

int claire_div(claire_ctx *ctx, const float *v, float *out) {
    API_BEGIN(ctx)
    need(v, "v");
    need(out, "out");
    ctx->div(v, out);
    check_launch("div");
    API_END(ctx)
}

int claire_apply_A(claire_ctx *ctx, const float *v, float *out) {
    API_BEGIN(ctx)
    need(v, "v");
    need(out, "out");
    ctx->spectral(OP_A, v, out, nullptr);
    check_launch("apply_A");
    API_END(ctx)
}

int claire_interp(claire_ctx *ctx, const float *f, const float *disp, float *out) {
    API_BEGIN(ctx)
    need(f, "f");
    need(disp, "disp");
    need(out, "out");
    if (f == out) throw Error(CLAIRE_ERR_ARG, "f and out may not alias");
    launch_interp(ctx->d, f, disp, out, ctx->rng_i(), ctx->st, &ctx->prof, CLAIRE_K_INTERP);
    check_launch("interp");
    API_END(ctx)
}

int claire_get_field(claire_ctx *ctx, int which, int j, float *out) {
    API_BEGIN(ctx)
    need(out, "out");
    const size_t N = ctx->d.N;
    const float *src = nullptr;
    size_t n = N;
    const bool hist = (which == CLAIRE_FIELD_STATE || which == CLAIRE_FIELD_GRADM ||
                       which == CLAIRE_FIELD_ADJ || which == CLAIRE_FIELD_INCADJ);
    if (hist && (j < 0 || j > ctx->nt)) throw Error(CLAIRE_ERR_ARG, "time index out of range");
    if (which != CLAIRE_FIELD_ADJ && which != CLAIRE_FIELD_INCADJ && which != CLAIRE_FIELD_INCST &&
        !ctx->have_lin)
        throw Error(CLAIRE_ERR_STATE, "no linearization");
    if (ctx->h16 && (which == CLAIRE_FIELD_STATE || which == CLAIRE_FIELD_GRADM || which == CLAIRE_FIELD_ADJ)) {
        const __half *h = which == CLAIRE_FIELD_STATE ? ctx->hist(ctx->mhist_h, j)
                        : which == CLAIRE_FIELD_GRADM ? ctx->hist(ctx->gmhist_h, j, 3)
                                                      : ctx->hist(ctx->lhist_h, j);
        launch_h2f(h, out, which == CLAIRE_FIELD_GRADM ? 3 * (long long)N : (long long)N, ctx->st, nullptr);
        check_launch("get_field");
        return CLAIRE_OK;
    }
    switch (which) {
        case CLAIRE_FIELD_DISPM: src = ctx->dispm; n = 3 * N; break;
        case CLAIRE_FIELD_DISPP: src = ctx->dispp; n = 3 * N; break;
        case CLAIRE_FIELD_STATE: src = ctx->hist(ctx->mhist, j); break;
        case CLAIRE_FIELD_GRADM: src = ctx->hist(ctx->gmhist, j, 3); n = 3 * N; break;
        case CLAIRE_FIELD_DIVV: src = ctx->divv; break;
        case CLAIRE_FIELD_ADJF: src = ctx->cfac; break;
        case CLAIRE_FIELD_ADJ:
        case CLAIRE_FIELD_INCADJ: src = ctx->hist(ctx->lhist, j); break;
        case CLAIRE_FIELD_INCST: src = ctx->mt; break;
        default: throw Error(CLAIRE_ERR_ARG, "unknown field");
    }
    CK(cudaMemcpyAsync(out, src, n * sizeof(float), cudaMemcpyDeviceToDevice, ctx->st));
    API_END(ctx)
}

void claire_solve_opts_default(claire_solve_opts *o) {
    if (!o) return;
    o->max_gn = 50;
    o->max_pcg = 100;
    o->fixed_pcg = 0;
    o->eps_n = 5e-2;
    o->armijo_c1 = 1e-4;
    o->max_ls = 12;
    o->precond = CLAIRE_PC_INVA;
    o->eps_h0 = 1e-3;
    o->max_inner = 500;
}

namespace {
struct EvTimer {
    cudaEvent_t a{}, b{};
    cudaStream_t st;
    double *acc;
    EvTimer(cudaStream_t s, double *acc_) : st(s), acc(acc_) {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, st);
    }
    ~EvTimer() {
        float ms = 0;
        cudaEventRecord(b, st);
        cudaEventSynchronize(b);
        cudaEventElapsedTime(&ms, a, b);
        *acc += ms;
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
};
}  // namespace

// One Gauss-Newton-Krylov solve (Algorithm 1) at the context's beta; returns
// CLAIRE_OK, CLAIRE_ERR_LINESEARCH or CLAIRE_ERR_NONFINITE (v then holds the
// last accepted iterate); other failures throw.
// v_host (optional): host buffer that receives the result.  Each accepted
// step's v is copied there on the auxiliary stream while the gradient at
// the new v runs (the last such copy is the result); the main stream waits
// for a copy to finish before it overwrites v again.
static int do_solve(claire_ctx *ctx, float *v, const claire_solve_opts &o, claire_solve_report *rep_out,
                    float *v_host = nullptr) {
    if (o.max_gn < 0 || o.max_pcg < 1 || o.fixed_pcg < 0 || !(o.eps_n >= 0) || o.max_ls < 0 ||
        o.precond < CLAIRE_PC_INVA || o.precond > CLAIRE_PC_2LINVH0 || !(o.eps_h0 > 0) || o.max_inner < 1)
        throw Error(CLAIRE_ERR_ARG, "invalid solve options");
    claire_solve_report rep;
    std::memset(&rep, 0, sizeof(rep));
    const long long n3 = 3 * ctx->d.N;
    // solver vectors; Av, Ax, Ap carry beta*A applied to v, the PCG iterate x
    // and the search direction p, so that no FFT is needed for them
    if (!ctx->sv) ctx->sv = ctx->alloc_f((size_t)10 * n3);
    float *g = ctx->sv, *x = g + n3, *r = x + n3, *z = r + n3, *p = z + n3, *q = p + n3, *vn = q + n3;
    float *Av = vn + n3, *Ax = Av + n3, *Ap = Ax + n3;
    const long long N = ctx->d.N;
    const double H3 = ctx->h3();
    cudaStream_t st = ctx->st;
    bool exported = false;  // a copy of the current v to v_host is issued
    auto export_v = [&]() {
        if (!v_host) return;
        CK(cudaEventRecord(ctx->ev_main, st));
        CK(cudaStreamWaitEvent(ctx->aux, ctx->ev_main, 0));
        CK(cudaMemcpyAsync(v_host, v, n3 * sizeof(float), cudaMemcpyDeviceToHost, ctx->aux));
        CK(cudaEventRecord(ctx->ev_vout, ctx->aux));
        exported = true;
    };
    // the copy out must end before v is overwritten, and before returning
    struct VoutWait {
        claire_ctx *c;
        const bool *on;
        ~VoutWait() {
            if (*on) cudaEventSynchronize(c->ev_vout);
        }
    } vout_wait{ctx, &exported};
    cudaEvent_t ev0, ev1;
    CK(cudaEventCreate(&ev0));
    CK(cudaEventCreate(&ev1));
    struct EvFree {
        cudaEvent_t a, b;
        ~EvFree() { cudaEventDestroy(a); cudaEventDestroy(b); }
    } evfree{ev0, ev1};
    CK(cudaEventRecord(ev0, st));
    ctx->gm0_valid = false;  // grad m0 is computed once per solve
    double J = 0;
    {
        Nvtx nv("gradient");
        EvTimer t(st, &rep.t_grad_ms);
        ctx->spectral(OP_A, v, Av, nullptr);
        ctx->gradient(v, g, &J, nullptr, Av);
    }
    const double g0 = std::sqrt(ctx->fetch(9));  // g . g from the gradient's last pass
    // a non-finite start (e.g. a NaN image) ends the solve with its report
    // filled and v as it came in, like a non-finite gradient later on
    int status = (std::isfinite(g0) && std::isfinite(J)) ? CLAIRE_OK : CLAIRE_ERR_NONFINITE;
    rep.J0 = J;
    rep.g0 = g0;
    double gn = g0;
    double vAv = ctx->last_vAv;  // <v, beta A v> (sum over the grid)
    int k = 0;
    while (status == CLAIRE_OK) {
        const double grel = g0 > 0 ? gn / g0 : 0.0;
        if (grel <= o.eps_n || k >= o.max_gn) break;
        const double epsk = std::fmin(std::sqrt(grel), 0.5);
        // ---- PCG on H x = -g, x0 = 0
        double t_pcg = 0;
        {
            Nvtx nv("pcg");
            EvTimer tp(st, &t_pcg);
            CK(cudaMemsetAsync(x, 0, n3 * sizeof(float), st));
            CK(cudaMemsetAsync(Ax, 0, n3 * sizeof(float), st));
            launch_axpby(r, -1.f, g, 0.f, nullptr, n3, st, &ctx->prof);
            launch_stats(r, N, ctx->partial, ctx->dres, st, &ctx->prof);
            const double r0 = std::sqrt(ctx->fetch(0));
            const int maxit = o.fixed_pcg > 0 ? o.fixed_pcg : o.max_pcg;
            int it = 0;
            // preconditioner z = M r; Az = beta*A z (NULL: the recurrence holds)
            auto apply_pc = [&]() -> const float * {
                Nvtx nv("precond");
                EvTimer t(st, &rep.t_pc_ms);
                rep.n_precond++;
                if (o.precond == CLAIRE_PC_INVA) {
                    ctx->spectral(OP_AINV, r, z, nullptr);
                    return nullptr;
                }
                if (o.precond == CLAIRE_PC_INVH0)
                    rep.n_inner += ctx->invh0(r, z, o.eps_h0 * epsk, o.max_inner, false);
                else
                    rep.n_inner += ctx->invh0_2l(r, z, o.eps_h0 * epsk, o.max_inner, false);
                ctx->spectral(OP_A, z, q, nullptr);
                return q;
            };
            // the direction update also writes u0 of the next matvec into s1a
            // and p . beta A p into dres[8] (the matvec's PCG form)
            // init: b = 0; otherwise b = dres[bn] / dres[bd] on the device
            auto pcg_dir = [&](const float *Az, bool init, int bn, int bd) {
                const float hdt = 0.5f / ctx->nt;
                const double *dbn = init ? nullptr : ctx->dres + bn, *dbd = init ? nullptr : ctx->dres + bd;
                if (ctx->h16)
                    launch_pcg_dir_u0(p, Ap, z, r, ctx->dres + 1, Az, 0.f, N, init, ctx->hist(ctx->gmhist_h, 0, 3),
                                      ctx->s1a, hdt, ctx->partial, ctx->dres + 8, st, &ctx->prof, dbn, dbd);
                else
                    launch_pcg_dir_u0(p, Ap, z, r, ctx->dres + 1, Az, 0.f, N, init, ctx->hist(ctx->gmhist, 0, 3),
                                      ctx->s1a, hdt, ctx->partial, ctx->dres + 8, st, &ctx->prof, dbn, dbd);
            };
            // The scalars of the recurrence stay on the device: r . z of the
            // current direction in dres[rz] (slots 10 and 11 in turn), p . Hp
            // in dres[0] from the matvec; the update takes alpha = rz / pq and
            // the direction update beta = rz_new / rz from there.  One host
            // read per iteration (r . r for the stopping test, p . Hp kept in
            // dres[12] for the curvature test) instead of three.
            // the loop as a graph (InvA, a stream that can be captured, the
            // profiler off): one launch and one host read per GN step
            auto pcg_graph = [&](int &iters) -> bool {
                claire_ctx &c = *ctx;
                if (!c.octl) c.octl = (double *)c.alloc_bytes(16 * sizeof(double));
                const bool fixed = o.fixed_pcg > 0;
                int slot = -1;
                for (int i = 0; i < 2; ++i) {
                    const auto &e = c.pgr[i];
                    if (e.exec && e.dispm == c.dispm && e.rng == c.rng_m() && e.sv == c.sv && e.maxit == maxit &&
                        e.fixed == fixed && e.beta == c.beta && e.gamma == c.gamma && e.iorder == c.d.iorder)
                        slot = i;
                }
                if (slot < 0) {
                    // replace the least recently used variant
                    slot = c.pgr[0].used <= c.pgr[1].used ? 0 : 1;
                    auto &e = c.pgr[slot];
                    if (e.exec) cudaGraphExecDestroy(e.exec);
                    e.exec = nullptr;
                    long ks = 0;
                    const bool ok = c.build_loop_graph(
                        &e.exec, [] {}, false,
                        [&](cudaGraphConditionalHandle h, cudaGraphConditionalHandle ht) {
                            c.matvec_launches(p, q, true);
                            launch_pcg_update(x, Ax, r, p, Ap, q, 0.f, N, c.partial, c.dres, st, &c.prof, true,
                                              c.dres, c.dres + 10, c.dres + 12);
                            launch_pcg_ctl(c.dres, c.octl, h, ht, maxit, fixed, st, &c.prof);
                            launch_pcg_negcopy(c.octl, x, Ax, z, Ap, n3, st, &c.prof);
                        },
                        [&] {
                            c.spectral(OP_AINV, r, z, nullptr);
                            launch_dot(r, z, n3, c.partial, c.dres + 11, st, &c.prof);
                            pcg_dir(nullptr, false, 11, 10);
                            launch_scalar_copy(c.dres + 10, c.dres + 11, st, &c.prof);
                        },
                        ks, e.k_head, e.k_tail);
                    if (!ok) {
                        c.pcg_graphs = false;
                        return false;
                    }
                    e.dispm = c.dispm; e.rng = c.rng_m(); e.sv = c.sv; e.maxit = maxit; e.fixed = fixed;
                    e.beta = c.beta; e.gamma = c.gamma; e.iorder = c.d.iorder;
                }
                auto &e = c.pgr[slot];
                e.used = ++c.pgr_clock;
                launch_pcg_ctl_init(c.octl, epsk * r0, st, &c.prof);
                CK(cudaGraphLaunch(e.exec, st));
                check_launch("pcg graph");
                double hc[4];
                CK(cudaMemcpyAsync(hc, c.octl, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
                // every loop body runs the head, all but the last one the tail
                c.prof.launches += (long)hc[3] * e.k_head + std::max(0L, (long)hc[3] - 1) * e.k_tail;
                if (hc[2] == 1.0) throw Error(CLAIRE_ERR_NONFINITE, "non-finite p.Hp in PCG");
                iters = (int)hc[1];
                return true;
            };
            if (r0 > 0) {
                const float *Az = apply_pc();
                pcg_dir(Az, true, 0, 0);
                int rz = 10;
                launch_dot(r, z, n3, ctx->partial, ctx->dres + rz, st, &ctx->prof);
                const bool use_graph = o.precond == CLAIRE_PC_INVA && ctx->pcg_graphs && ctx->use_graphs &&
                                       claire_ctx::capturable(st) && !ctx->prof.on;
                int git = 0;
                const bool by_graph = use_graph && pcg_graph(git);
                if (by_graph) {
                    it = git;
                    rep.n_matvec += it;
                    rep.n_precond += it - 1;  // the first one is counted above
                }
                while (!by_graph && it < maxit) {
                    {
                        Nvtx nv("hess_matvec");
                        EvTimer t(st, &rep.t_hess_ms);
                        ctx->matvec(p, q, true);
                    }
                    rep.n_matvec++;
                    // x, Ax, r change only when p . Hp > 0
                    launch_pcg_update(x, Ax, r, p, Ap, q, 0.f, N, ctx->partial, ctx->dres, st, &ctx->prof, true,
                                      ctx->dres, ctx->dres + rz, ctx->dres + 12);
                    double h[13];
                    ctx->fetch_n(0, 13, h);
                    const double pq = h[12];
                    if (!std::isfinite(pq)) throw Error(CLAIRE_ERR_NONFINITE, "non-finite p.Hp in PCG");
                    if (pq <= 0) {
                        if (it == 0) {
                            // keep the preconditioned residual z0 = p0 (and beta*A z0 = Ap0)
                            CK(cudaMemcpyAsync(x, z, n3 * sizeof(float), cudaMemcpyDeviceToDevice, st));
                            CK(cudaMemcpyAsync(Ax, Ap, n3 * sizeof(float), cudaMemcpyDeviceToDevice, st));
                        }
                        ++it;
                        break;
                    }
                    ++it;
                    const double rn = std::sqrt(h[0]);
                    if (o.fixed_pcg == 0 && rn <= epsk * r0) break;
                    if (it >= maxit) break;
                    const float *Az = apply_pc();
                    const int rz_new = 21 - rz;
                    launch_dot(r, z, n3, ctx->partial, ctx->dres + rz_new, st, &ctx->prof);
                    pcg_dir(Az, false, rz_new, rz);
                    rz = rz_new;
                }
            }
            rep.n_pcg += it;
        }
        rep.t_pcg_ms += t_pcg;
        // ---- Armijo backtracking; the regularization term of J(v + a x) is
        // 1/2 <v + a x, Av + a Ax>, a quadratic in a from three dot products
        launch_ls_dots(g, x, Av, v, Ax, n3, ctx->partial, ctx->dres, st, &ctx->prof);
        double lsd[4];
        ctx->fetch_n(0, 4, lsd);
        const double slope = H3 * lsd[0];
        const double xAv = lsd[1], vAx = lsd[2], xAx = lsd[3];
        double alpha = 1.0;
        bool ok = false;
        {
            Nvtx nv("line_search");
            EvTimer t(st, &rep.t_obj_ms);
            for (int ls = 0; ls <= o.max_ls; ++ls) {
                launch_axpby(vn, 1.f, v, (float)alpha, x, n3, st, &ctx->prof);
                const double mis = ctx->trial_mismatch(vn);
                const double reg = 0.5 * H3 * (vAv + alpha * (xAv + vAx) + alpha * alpha * xAx);
                const double Jt = mis + reg;
                rep.n_ls++;
                if (std::isfinite(Jt) && Jt <= J + o.armijo_c1 * alpha * slope) {
                    ok = true;
                    break;
                }
                alpha *= 0.5;
            }
        }
        if (!ok) {
            status = CLAIRE_ERR_LINESEARCH;
            break;
        }
        if (exported) CK(cudaStreamWaitEvent(st, ctx->ev_vout, 0));
        CK(cudaMemcpyAsync(v, vn, n3 * sizeof(float), cudaMemcpyDeviceToDevice, st));
        export_v();
        launch_axpby(Av, 1.f, Av, (float)alpha, Ax, n3, st, &ctx->prof);
        if (ctx->keeps_trial()) ctx->adopt_trial();
        ++k;
        {
            Nvtx nv("gradient");
            EvTimer t(st, &rep.t_grad_ms);
            ctx->gradient(v, g, &J, nullptr, Av, ctx->keeps_trial());
        }
        vAv = ctx->last_vAv;
        gn = std::sqrt(ctx->fetch(9));
        if (!std::isfinite(gn) || !std::isfinite(J)) {
            status = CLAIRE_ERR_NONFINITE;
            break;
        }
    }
    rep.n_gn = k;
    rep.J = J;
    rep.g = gn;
    rep.grel = g0 > 0 ? gn / g0 : 0.0;
    {
        // relative mismatch at the final v: the cached state is at v
        const double a = ctx->final_mismatch() / (0.5 * ctx->h3());
        launch_sqdiff(ctx->m0, ctx->m1, ctx->d.N, ctx->partial, ctx->dres, st, &ctx->prof);
        const double b = ctx->fetch();
        rep.mismatch_rel = b > 0 ? std::sqrt(a / b) : 0.0;
    }
    if (v_host && !exported) export_v();  // no accepted step: v as it came in
    rep.status = status;
    {
        float ms = 0;
        CK(cudaEventRecord(ev1, st));
        CK(cudaEventSynchronize(ev1));
        CK(cudaEventElapsedTime(&ms, ev0, ev1));
        rep.t_total_ms = ms;
    }
    if (rep_out) *rep_out = rep;
    if (status != CLAIRE_OK)
        ctx->err = status == CLAIRE_ERR_LINESEARCH ? "line search failed" : "non-finite gradient";
    return status;
}

int claire_solve(claire_ctx *ctx, float *v, const claire_solve_opts *opts, claire_solve_report *rep_out) {
    API_BEGIN(ctx)
    need(v, "v_inout");
    claire_solve_opts o;
    if (opts) o = *opts; else claire_solve_opts_default(&o);
    const int status = do_solve(ctx, v, o, rep_out);
    if (status != CLAIRE_OK) return status;
    API_END(ctx)
}

int claire_solve_host(claire_ctx *ctx, const float *m0, const float *m1, const float *v_in, float *v_out,
                      const claire_solve_opts *opts, claire_solve_report *rep_out) {
    API_BEGIN(ctx)
    need(m0, "m0");
    need(m1, "m1");
    need(v_in, "v_in");
    need(v_out, "v_out");
    claire_solve_opts o;
    if (opts) o = *opts; else claire_solve_opts_default(&o);
    ctx->ensure_aux();
    const long long N = ctx->d.N;
    if (!ctx->vdev) ctx->vdev = ctx->alloc_f((size_t)3 * N);
    // the images go in on the auxiliary stream once the work already queued
    // on the context's stream (which may read the old images) is done; v on
    // the main stream meanwhile; the solve waits for the images only where it
    // first reads them, after its first foot points
    CK(cudaEventRecord(ctx->ev_main, ctx->st));
    CK(cudaStreamWaitEvent(ctx->aux, ctx->ev_main, 0));
    CK(cudaMemcpyAsync(ctx->m0, m0, N * sizeof(float), cudaMemcpyHostToDevice, ctx->aux));
    CK(cudaMemcpyAsync(ctx->m1, m1, N * sizeof(float), cudaMemcpyHostToDevice, ctx->aux));
    CK(cudaEventRecord(ctx->ev_img, ctx->aux));
    ctx->img_pending = true;
    ctx->have_images = true;
    ctx->have_lin = false;
    ctx->gm0_valid = false;
    struct ImgWait {
        claire_ctx *c;
        ~ImgWait() { c->wait_images(); }
    } img_wait{ctx};
    CK(cudaMemcpyAsync(ctx->vdev, v_in, 3 * N * sizeof(float), cudaMemcpyHostToDevice, ctx->st));
    const int status = do_solve(ctx, ctx->vdev, o, rep_out, v_out);
    if (status != CLAIRE_OK) return status;
    API_END(ctx)
}

// host threads (and streams) of a batch solve
constexpr int kBatchWorkers = 8;

int claire_solve_batch(claire_ctx *const *ctxs, float *const *v, int n, const claire_solve_opts *opts,
                       claire_solve_report *reports) {
    if (!ctxs || !v || n < 1 || n > 1024) {
        set_thread_error("claire_solve_batch: need n in [1, 1024] and non-NULL arrays");
        return CLAIRE_ERR_ARG;
    }
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i] || !v[i]) {
            set_thread_error("claire_solve_batch: NULL context or velocity");
            return CLAIRE_ERR_ARG;
        }
        for (int k = 0; k < i; ++k)
            if (ctxs[k] == ctxs[i]) {
                set_thread_error("claire_solve_batch: a context appears twice");
                return CLAIRE_ERR_ARG;
            }
    }
    claire_solve_opts o;
    if (opts) o = *opts; else claire_solve_opts_default(&o);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        set_thread_error("claire_solve_batch: no current device");
        return CLAIRE_ERR_CUDA;
    }
    // each registration runs on a stream of its own, driven by a host thread
    // of its own (its PCG and line search branch on its own FP64 scalars);
    // the hardware interleaves the kernels of the streams
    std::vector<cudaStream_t> own(n, nullptr), prev(n, nullptr);
    std::vector<int> status(n, CLAIRE_OK);
    int rc = CLAIRE_OK;
    for (int i = 0; i < n && rc == CLAIRE_OK; ++i) {
        prev[i] = ctxs[i]->st;
        if (cudaStreamSynchronize(prev[i]) != cudaSuccess ||
            (i < kBatchWorkers && cudaStreamCreateWithFlags(&own[i], cudaStreamNonBlocking) != cudaSuccess)) {
            ctxs[i]->err = "claire_solve_batch: stream setup failed";
            rc = CLAIRE_ERR_CUDA;
        }
    }
    if (reports) std::memset(reports, 0, (size_t)n * sizeof(claire_solve_report));
    if (rc == CLAIRE_OK) {
        // Workers (host threads, one stream each) take the registrations
        // largest grid first from a shared counter; each registration runs the
        // plain solve on its worker's stream (its PCG and line search branch on
        // its own FP64 scalars) and the hardware interleaves the streams.
        // Eight workers and largest-first order measured 126 against 128 ms
        // for one stream per pair (16 pairs); the outer PCG loop stays
        // host-driven here: the conditional-node graphs measured slower with
        // several streams at once (137 ms at four or eight workers), while
        // they win one by one.
        const int nw = std::min(n, kBatchWorkers);
        std::vector<int> order(n);
        for (int i = 0; i < n; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return ctxs[a]->d.N > ctxs[b]->d.N; });
        std::atomic<int> next{0};
        std::vector<std::thread> th;
        th.reserve(nw);
        for (int w = 0; w < nw; ++w) {
            th.emplace_back([&, w] {
                cudaSetDevice(dev);
                for (;;) {
                    const int q = next.fetch_add(1);
                    if (q >= n) break;
                    const int i = order[q];
                    claire_ctx *c = ctxs[i];
                    c->st = own[w];
                    const bool pg = c->pcg_graphs;
                    c->pcg_graphs = false;
                    try {
                        status[i] = do_solve(c, v[i], o, reports ? &reports[i] : nullptr);
                    } catch (const Error &e) {
                        c->err = e.msg;
                        status[i] = e.code;
                    } catch (const std::bad_alloc &) {
                        c->err = "host allocation failed";
                        status[i] = CLAIRE_ERR_OOM;
                    } catch (const std::exception &e) {
                        c->err = e.what();
                        status[i] = CLAIRE_ERR_CUDA;
                    }
                    c->pcg_graphs = pg;
                    if (reports && status[i] != CLAIRE_OK) reports[i].status = status[i];
                }
            });
        }
        for (auto &t : th) t.join();
        for (int i = 0; i < n; ++i)
            if (status[i] != CLAIRE_OK && rc == CLAIRE_OK) rc = status[i];
    }
    for (int i = 0; i < n; ++i) {
        if (own[i]) {
            cudaStreamSynchronize(own[i]);
            cudaStreamDestroy(own[i]);
        }
        ctxs[i]->st = prev[i];
    }
    return rc;
}

int claire_solve_continuation(claire_ctx *ctx, float *v, double beta_target, double beta_start,
                              double factor, const claire_solve_opts *opts,
                              claire_solve_report *rep_out, int *levels) {
    API_BEGIN(ctx)
    need(v, "v_inout");
    check_params(beta_target, ctx->gamma);
    if (!(beta_start > 0) || !std::isfinite(beta_start) || !(factor > 0 && factor < 1))
        throw Error(CLAIRE_ERR_ARG, "need beta_start > 0 and 0 < factor < 1");
    claire_solve_opts o;
    if (opts) o = *opts; else claire_solve_opts_default(&o);
    claire_solve_report acc, r;
    std::memset(&acc, 0, sizeof(acc));
    double b = beta_start > beta_target ? beta_start : beta_target;
    int nlev = 0, status = CLAIRE_OK;
    for (;;) {
        claire_solve_opts ol = o;
        if (b > 5e-1) ol.precond = CLAIRE_PC_INVA;  // spectral preconditioner for large beta
        ctx->beta = b;
        ctx->have_lin = false;
        std::memset(&r, 0, sizeof(r));
        status = do_solve(ctx, v, ol, &r);
        ++nlev;
        acc.n_gn += r.n_gn;
        acc.n_pcg += r.n_pcg;
        acc.n_matvec += r.n_matvec;
        acc.n_precond += r.n_precond;
        acc.n_ls += r.n_ls;
        acc.n_inner += r.n_inner;
        acc.t_grad_ms += r.t_grad_ms;
        acc.t_hess_ms += r.t_hess_ms;
        acc.t_pc_ms += r.t_pc_ms;
        acc.t_obj_ms += r.t_obj_ms;
        acc.t_pcg_ms += r.t_pcg_ms;
        acc.t_total_ms += r.t_total_ms;
        if (nlev == 1) {
            acc.J0 = r.J0;
            acc.g0 = r.g0;
        }
        acc.J = r.J;
        acc.g = r.g;
        acc.grel = r.grel;
        acc.mismatch_rel = r.mismatch_rel;
        if (status != CLAIRE_OK || b <= beta_target) break;
        b *= factor;
        if (b <= beta_target * (1.0 + 1e-9)) b = beta_target;  // land exactly on the target
    }
    acc.status = status;
    ctx->beta = beta_target;
    if (rep_out) *rep_out = acc;
    if (levels) *levels = nlev;
    if (status != CLAIRE_OK) return status;
    API_END(ctx)
}

int claire_profile_enable(claire_ctx *ctx, int on) {
    API_BEGIN(ctx)
    ctx->prof.on = on != 0;
    ctx->prof.reset();
    API_END(ctx)
}

int claire_profile_read(claire_ctx *ctx, int cls, long *launches, double *total_ms,
                        double *total_bytes) {
    API_BEGIN(ctx)
    if (cls < 0 || cls >= CLAIRE_K_COUNT) throw Error(CLAIRE_ERR_ARG, "kernel class out of range");
    CK(cudaStreamSynchronize(ctx->st));
    long n = 0;
    double ms = 0, by = 0;
    for (size_t i = 0; i < ctx->prof.used; ++i) {
        auto &r = ctx->prof.recs[i];
        if (r.cls != cls) continue;
        float t = 0;
        CK(cudaEventElapsedTime(&t, r.a, r.b));
        ms += t;
        by += r.bytes;
        ++n;
    }
    if (launches) *launches = n;
    if (total_ms) *total_ms = ms;
    if (total_bytes) *total_bytes = by;
    API_END(ctx)
}

int claire_launch_count(const claire_ctx *ctx, long *launches) {
    if (!ctx || !launches) return CLAIRE_ERR_ARG;
    *launches = ctx->prof.launches;
    return CLAIRE_OK;
}

int claire_set_workspace_limit(size_t bytes) {
    g_workspace_limit.store(bytes);
    return CLAIRE_OK;
}

int claire_workspace_bytes(const claire_ctx *ctx, size_t *bytes) {
    if (!ctx || !bytes) return CLAIRE_ERR_ARG;
    *bytes = ctx->bytes;
    return CLAIRE_OK;
}

const char *claire_last_error(const claire_ctx *ctx) {
    if (!ctx) return g_create_error.c_str();
    return ctx->err.c_str();
}

}  // extern "C"
