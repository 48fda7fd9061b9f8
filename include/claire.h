/*
 * claire.h -- C ABI of the GB300 (sm_103a) Gauss-Newton-Krylov diffeomorphic
 * registration library, after Brunn, Himthani, Biros, Mehl and Mang,
 * "Multi-Node Multi-GPU Diffeomorphic Image Registration for Large-Scale
 * Imaging Problems" (arXiv 2008.12820).
 *
 * The problem (paper Section 2.1, Eq. 2.1): find a stationary velocity v on
 * the periodic domain Omega = [0, 2*pi)^3 minimizing
 *     J(v) = 1/2 ||m(., 1) - m1||^2_{L2} + 1/2 <beta*A v, v>_{L2}
 * subject to the transport equation d_t m + v . grad m = 0, m(., 0) = m0.
 * beta*A is the vector Laplacian (H1 seminorm) augmented with a divergence
 * penalty: beta*A = -beta * Laplace - gamma * grad div.
 *
 * Conventions shared by every call
 * ---------------------------------
 * Grid: nx * ny * nz points, x_ijk = (i*hx, j*hy, k*hz), h = 2*pi/n per axis.
 *   A scalar field is float[nx][ny][nz] (z contiguous); a vector field is
 *   three scalar fields one after another, float[3][nx][ny][nz].  Velocities
 *   are in domain units per unit time.  N = nx*ny*nz.
 * Memory: every field pointer is DEVICE memory owned by the caller, 4-byte
 *   aligned (16-byte alignment is faster), never retained past the call
 *   (claire_set_images copies).  The context owns all workspace (allocated in
 *   claire_create with cudaMalloc) and a cached linearization at the last v
 *   given to claire_gradient / claire_linearize.
 * Streams: all work is ordered on the context's stream (claire_set_stream;
 *   default: the legacy default stream).  A call that returns a host scalar
 *   synchronizes that stream before returning; other calls return as soon as
 *   the work is enqueued.
 * Errors: every call returns a claire_status.  On error the outputs are
 *   unspecified, the context stays usable, and claire_last_error() gives a
 *   message.  No C++ exception crosses this boundary.
 * Threads: a context may be used by one host thread at a time.
 * Inner products: <a, b>_{L2} is the sum over grid points times hx*hy*hz.
 *   g below is the L2 (Riesz) gradient; the Euclidean gradient of the
 *   discrete J is hx*hy*hz * g.
 */
#ifndef CLAIRE_H
#define CLAIRE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct claire_ctx claire_ctx;

typedef enum {
    CLAIRE_OK = 0,
    CLAIRE_ERR_ARG = 1,          /* invalid argument (size, null pointer, parameter) */
    CLAIRE_ERR_OOM = 2,          /* device allocation failed */
    CLAIRE_ERR_CUDA = 3,         /* a CUDA call or kernel launch failed */
    CLAIRE_ERR_STATE = 4,        /* call order violated (e.g. no images set) */
    CLAIRE_ERR_NONFINITE = 5,    /* NaN/Inf detected in a gradient, objective or PCG scalar */
    CLAIRE_ERR_LINESEARCH = 6,   /* Armijo line search found no acceptable step */
    CLAIRE_ERR_PCG_BREAKDOWN = 7,/* PCG curvature p.Hp <= 0 (reported, not fatal in solve) */
    CLAIRE_ERR_TIMEOUT = 8       /* a bounded device wait gave up */
} claire_status;

/* Create a context for an nx*ny*nz grid with nt semi-Lagrangian time steps
 * (dt = 1/nt), regularization weight beta > 0 and divergence penalty
 * gamma >= 0 (paper Section 2.1, Eq. 2.1; Section 3 "Discretization").
 * Each n must be in [4, 1024] and a product of powers of 2, 3 and 5 (the
 * pencil FFT radices); nt in [1, 256].  Allocates all device workspace on the
 * current device.  *out receives the context or NULL on error. */
int claire_create(int nx, int ny, int nz, int nt, double beta, double gamma, claire_ctx **out);

/* Precision of the stored trajectories.  CLAIRE_PREC_FP32: everything FP32
 * (the paper's setting).  CLAIRE_PREC_FP16_STORAGE: the state trajectory m^j,
 * its gradient grad m^j and the gradient's adjoint lambda^j (j = 0..nt) are
 * stored in FP16 (IEEE binary16, round to nearest even on store) and widened
 * to FP32 on load; interpolation, spectral operators and body-force
 * accumulation run in FP32, reductions in FP64 as in the FP32 form.  The
 * incremental state and adjoint of the Hessian matvec stay FP32 (their scale
 * follows the PCG direction, which FP16's range does not cover).  The paper
 * has no FP16 form; results differ from the FP32 form by the FP16 rounding
 * of the stored fields (about 5e-4 relative per stored value). */
enum { CLAIRE_PREC_FP32 = 0, CLAIRE_PREC_FP16_STORAGE = 1 };

/* claire_create with a precision mode (CLAIRE_PREC_*); claire_create is
 * claire_create_ex(..., CLAIRE_PREC_FP32, out).  An unknown mode is
 * CLAIRE_ERR_ARG. */
int claire_create_ex(int nx, int ny, int nz, int nt, double beta, double gamma, int precision,
                     claire_ctx **out);

/* Release the context and its device memory (NULL is a no-op). */
int claire_destroy(claire_ctx *ctx);

/* Order all later work of ctx on `stream` (a cudaStream_t; NULL = legacy). */
int claire_set_stream(claire_ctx *ctx, void *stream);

/* Change beta and gamma (same rules as claire_create); drops nothing but the
 * cached gradient/objective values. */
int claire_set_params(claire_ctx *ctx, double beta, double gamma);

/* Discretization (Sections 4.1 and 4.2): interp_order 3 = periodic cubic
 * Lagrange interpolation (default), 1 = trilinear; deriv
 * CLAIRE_DERIV_SPECTRAL (default) or CLAIRE_DERIV_FD8 (eighth-order central
 * differences) for the first derivatives grad m and div v -- the paper's GPU
 * configuration is trilinear with FD8.  The regularization operator and its
 * inverse stay spectral.  claire_grad and claire_div follow the setting.
 * Invalidates the cached linearization. */
enum { CLAIRE_DERIV_SPECTRAL = 0, CLAIRE_DERIV_FD8 = 1 };
int claire_set_discretization(claire_ctx *ctx, int interp_order, int deriv);

/* Copy template m0 and reference m1 (device, float[N] each) into ctx.
 * Invalidates the cached linearization. */
int claire_set_images(claire_ctx *ctx, const float *m0, const float *m1);

/* Forward problem (Eq. 2.1b by the semi-Lagrangian scheme of Section 3):
 * m(.,1) from m0 along the RK2 backward characteristics of v (float[3][N]).
 * Writes m(.,1) to m_final (float[N], nullable) and
 * *mismatch = 1/2 ||m(.,1) - m1||^2_{L2} (nullable; synchronizes if given).
 * Does not touch the cached linearization. */
int claire_forward(claire_ctx *ctx, const float *v, float *m_final, double *mismatch);

/* Differentiable forward (Eq. 2.1b): m(1) from m0 along the characteristics
 * of v, keeping the state only every checkpoint_stride time steps (and at
 * t = 1); *mismatch = 1/2 ||m(1) - m1||^2_{L2} (nullable; synchronizes).
 * m_final: float[N] (nullable).  checkpoint_stride in [1, nt], or 0: chosen
 * from the memory left on the device (and under claire_set_workspace_limit)
 * -- every state kept (stride 1: the backward recomputes nothing) when that
 * fits, else the stride that needs the least memory (CLAIRE_ERR_OOM if none
 * fits).  The first call fixes the stride of ctx (see
 * claire_checkpoint_stride).  Leaves the Gauss-Newton linearization
 * invalid.  The memory model follows the paper's Section 5 (the state history
 * dominates; keep it when it fits, recompute otherwise). */
int claire_mismatch_forward(claire_ctx *ctx, const float *v, float *m_final, double *mismatch,
                            int checkpoint_stride);

/* Checkpoint stride the differentiable form of ctx uses (0 before its first
 * claire_mismatch_forward). */
int claire_checkpoint_stride(const claire_ctx *ctx, int *stride);

/* Backward of the last claire_mismatch_forward (same v): the adjoint of
 * Eq. 3.2 from lambda(1) = grad_mismatch * (m1 - m(1)) - grad_m_final / h^3
 * (grad_m_final: float[N] upstream gradient of m(1), nullable), each segment
 * of the state recomputed from its checkpoint, and the body force
 * int lambda grad m dt by the trapezoidal rule.  Writes the Euclidean gradient
 * grad_v = hx*hy*hz * int lambda grad m dt (float[3][N]) of
 * grad_mismatch * mismatch + <grad_m_final, m(1)>. */
int claire_mismatch_backward(claire_ctx *ctx, double grad_mismatch, const float *grad_m_final,
                             float *grad_v);

/* Objective J(v) of Eq. 2.1a: mismatch term plus 1/2 <beta*A v, v>_{L2}.
 * Synchronizes. */
int claire_objective(claire_ctx *ctx, const float *v, double *objective, double *mismatch);

/* Linearize at v (float[3][N]): RK2 foot points X- and X+, the state history
 * m^j (j = 0..nt), its spectral gradients grad m^j (stored, paper Section 5.2),
 * div v and the adjoint source factor.  Cached for claire_hess_matvec. */
int claire_linearize(claire_ctx *ctx, const float *v);

/* Reduced gradient (Eq. 3.1): g = beta*A v + int_0^1 lambda grad m dt with
 * lambda from the adjoint equation (Eq. 3.2), lambda(1) = m1 - m(1).
 * Linearizes at v (cached).  g: float[3][N].  *objective (nullable; J of
 * Eq. 2.1a at v) synchronizes. */
int claire_gradient(claire_ctx *ctx, const float *v, float *g, double *objective);

/* Gauss-Newton Hessian matvec (Eq. 3.4): Hvt = beta*A vt + int lt grad m dt,
 * lt from the incremental adjoint (Eq. 3.6) with lt(1) = -mt(1), mt from the
 * incremental state (Eq. 3.5).  v is the linearization point: if v is NULL the
 * cached linearization is used (CLAIRE_ERR_STATE if there is none); otherwise
 * v is compared on the device with the cached point and the context
 * re-linearizes when they differ.  vt, Hvt: float[3][N] (may not alias). */
int claire_hess_matvec(claire_ctx *ctx, const float *v, const float *vt, float *Hvt);

/* Spectral preconditioner (Section 3 "Preconditioning"): s = (beta*A)^{-1} r,
 * identity on the zero wavenumber.  r, s: float[3][N]; s may equal r. */
int claire_precond(claire_ctx *ctx, const float *r, float *s);

/* Zero-velocity Hessian preconditioner InvH0 (Section 3 "Preconditioning",
 * Algorithm 2): s = H0^{-1} r with H0 = beta0 A + grad m (x) grad m, where
 * beta0 = max(beta, 5e-2) and grad m = grad m(., 1) of the cached
 * linearization (the deformed template at the current iterate).  Solved by
 * PCG preconditioned with (beta0 A)^{-1} from s = 0 until the residual drops
 * to tol times the initial one, or for exactly maxit iterations if tol == 0.
 * two_level != 0 selects the two-level variant: r and grad m are restricted
 * spectrally to the grid of half the resolution (wavenumbers |k_d| < n_d/4
 * kept), the system is solved there, and the prolonged solution is added to
 * the high-pass part of (beta0 A)^{-1} r (needs even sizes whose halves are
 * valid, >= 4).  r, s: float[3][N], distinct.  *iterations (nullable) gets
 * the (inner) iteration count.  CLAIRE_ERR_STATE without a linearization.
 * Synchronizes. */
int claire_precond_h0(claire_ctx *ctx, const float *r, float *s, double tol, int maxit,
                      int two_level, int *iterations);

/* ---- single operators (for checks and composition) ------------------- */

/* Gradient of a scalar field (Section 3): spectral, g_d = F^-1[i k_d F f],
 * or FD8 after claire_set_discretization.  f: float[N], g: float[3][N]. */
int claire_grad(claire_ctx *ctx, const float *f, float *g);

/* Divergence of a vector field: spectral, out = sum_d F^-1[i k_d F v_d], or
 * FD8 after claire_set_discretization. */
int claire_div(claire_ctx *ctx, const float *v, float *out);

/* beta*A applied to a vector field (Eq. 3.1 regularization term). */
int claire_apply_A(claire_ctx *ctx, const float *v, float *out);

/* Periodic cubic Lagrange interpolation (Section 4.1) of the scalar field f
 * at the points x_ijk + disp_ijk, disp: float[3][N] in grid-index units.
 * out: float[N]. */
int claire_interp(claire_ctx *ctx, const float *f, const float *disp, float *out);

/* Copy a part of the cached linearization into a caller buffer (float):
 *   CLAIRE_FIELD_DISPM  X- minus x, index units, [3][N]
 *   CLAIRE_FIELD_DISPP  X+ minus x, index units, [3][N]
 *   CLAIRE_FIELD_STATE  m^j, [N]            (j = 0..nt)
 *   CLAIRE_FIELD_GRADM  grad m^j, [3][N]    (j = 0..nt)
 *   CLAIRE_FIELD_DIVV   div v, [N]
 *   CLAIRE_FIELD_ADJF   adjoint factor c = 1 + dt/2 (d(X+) + d) + dt^2/2 d d(X+), [N]
 *   CLAIRE_FIELD_ADJ    lambda^j of the last gradient, [N] (j = 0..nt)
 *   CLAIRE_FIELD_INCADJ incremental adjoint lt^j of the last matvec, [N]
 *   CLAIRE_FIELD_INCST  mt(1) of the last matvec, [N]                    */
enum {
    CLAIRE_FIELD_DISPM = 0, CLAIRE_FIELD_DISPP = 1, CLAIRE_FIELD_STATE = 2,
    CLAIRE_FIELD_GRADM = 3, CLAIRE_FIELD_DIVV = 4, CLAIRE_FIELD_ADJF = 5,
    CLAIRE_FIELD_ADJ = 6, CLAIRE_FIELD_INCADJ = 7, CLAIRE_FIELD_INCST = 8
};
int claire_get_field(claire_ctx *ctx, int which, int j, float *out);

/* ---- Gauss-Newton-Krylov solver (Algorithm 1, Eq. 3.3) --------------- */

/* preconditioners of the Gauss-Newton system (Section 3 "Preconditioning") */
enum { CLAIRE_PC_INVA = 0, CLAIRE_PC_INVH0 = 1, CLAIRE_PC_2LINVH0 = 2 };

typedef struct {
    int max_gn;        /* max Gauss-Newton iterations (default 50) */
    int max_pcg;       /* max PCG iterations per GN step (default 100) */
    int fixed_pcg;     /* > 0: exactly this many PCG iterations per GN step */
    double eps_n;      /* stop when ||g_k|| / ||g_0|| <= eps_n (default 5e-2) */
    double armijo_c1;  /* sufficient decrease constant (default 1e-4) */
    int max_ls;        /* max step halvings in the line search (default 12) */
    int precond;       /* CLAIRE_PC_INVA (default), CLAIRE_PC_INVH0, CLAIRE_PC_2LINVH0 */
    double eps_h0;     /* InvH0 inner tolerance factor: inner tol = eps_h0 * eps_K (1e-3) */
    int max_inner;     /* max inner PCG iterations per InvH0 application (500) */
} claire_solve_opts;

typedef struct {
    int n_gn;          /* GN steps taken */
    int n_pcg;         /* PCG iterations over all GN steps */
    int n_matvec;      /* Hessian matvecs */
    int n_precond;     /* preconditioner applications */
    int n_ls;          /* objective evaluations in line searches */
    int status;        /* claire_status of the solve */
    double J0, J;      /* objective at the initial and final v */
    double g0, g;      /* ||g|| (2-norm over the grid) at the initial and final v */
    double grel;       /* g / g0 */
    double mismatch_rel; /* ||m(1) - m1|| / ||m0 - m1|| at the final v */
    long n_inner;      /* inner PCG iterations of InvH0 over the solve */
    /* CUDA-event times.  On a stream that can be captured, the PCG loop with
     * the InvA preconditioner runs as one CUDA graph (device-side stopping
     * test, one host read per Gauss-Newton step); its Hessian matvecs and
     * preconditioner applications are then inside t_pcg_ms and not split
     * out (t_hess_ms, t_pc_ms stay 0 for those loops). */
    double t_grad_ms, t_hess_ms, t_pc_ms, t_obj_ms, t_pcg_ms, t_total_ms;
} claire_solve_report;

/* Fill *opts with the defaults above. */
void claire_solve_opts_default(claire_solve_opts *opts);

/* Solve from the initial velocity in v_inout (device, float[3][N]); the
 * result overwrites it.  PCG: x0 = 0, r0 = -g, preconditioner (beta*A)^{-1},
 * forcing eps_K = min(sqrt(||g_k||/||g_0||), 0.5) (Algorithm 1), FP64 dot
 * products; stops at ||r|| <= eps_K ||r0||, max_pcg, or p.Hp <= 0 (keeps the
 * current iterate).  Armijo: alpha = 1, halve until
 * J(v + alpha vt) <= J(v) + c1 alpha <g, vt>_{L2}.  report may be NULL.
 * Returns CLAIRE_OK, or CLAIRE_ERR_LINESEARCH / CLAIRE_ERR_NONFINITE (v_inout
 * then holds the last accepted iterate, and the report is filled with the
 * status, e.g. a NaN in an image gives CLAIRE_ERR_NONFINITE with n_gn = 0). */
int claire_solve(claire_ctx *ctx, float *v_inout, const claire_solve_opts *opts,
                 claire_solve_report *report);

/* claire_set_images + claire_solve with HOST buffers, the host<->device
 * copies overlapped with the computation: m0, m1 (float[N] each), v_in (the
 * initial velocity) and v_out (the result; may be v_in) are host memory,
 * float[3][N] for the velocities.  The images are copied in on a second
 * stream while the first foot points (which need only v) run; each accepted
 * iterate is copied out while the gradient at it is computed, so the result
 * is in v_out when the call returns.  The results equal claire_set_images +
 * claire_solve on device copies, bit for bit.  Page-locked host memory is
 * needed for the copies to overlap (pageable memory works, without overlap).
 * The context keeps a device copy of v (12 B/voxel) from the first call on.
 * Errors: as claire_solve, plus CLAIRE_ERR_ARG for NULL pointers; v_out is
 * unspecified after an error other than CLAIRE_ERR_LINESEARCH /
 * CLAIRE_ERR_NONFINITE (which leave the last accepted iterate there). */
int claire_solve_host(claire_ctx *ctx, const float *m0, const float *m1, const float *v_in, float *v_out,
                      const claire_solve_opts *opts, claire_solve_report *report);

/* Batched form (no counterpart in the paper, which registers one pair at a
 * time): solve n independent registrations together, one per context, each
 * exactly as claire_solve would (same options for all; contexts may differ
 * in grid size, nt, beta, gamma and precision).  Up to eight host threads,
 * each with a CUDA stream created for the call, take the contexts largest
 * grid first and solve them one after the other on their stream, so the
 * kernels of different pairs overlap on the GPU; the results are bitwise
 * those of n claire_solve calls.  ctxs[i] (distinct, on the current device)
 * with velocity v[i] (float[3][N_i], device, in/out); reports may be NULL,
 * else n entries.  The call first synchronizes each context's stream and
 * restores it on return.  Returns CLAIRE_OK or the first failing status
 * (each report then holds its own; claire_last_error(ctxs[i]) the message);
 * n in [1, 1024] and NULL or repeated contexts are CLAIRE_ERR_ARG. */
int claire_solve_batch(claire_ctx *const *ctxs, float *const *v, int n,
                       const claire_solve_opts *opts, claire_solve_report *reports);

/* Parameter continuation in beta (Section 3 "Preconditioning", last
 * paragraph): Gauss-Newton solves for beta_k = max(beta_target,
 * beta_start * factor^k), k = 0, 1, ..., each started from the previous
 * velocity in v_inout.  Levels with beta_k > 5e-1 use the spectral
 * preconditioner, the others opts->precond.  The report accumulates the
 * counts and times of all levels and holds the last level's objective and
 * gradient values; *levels (nullable) gets the number of levels.  Leaves the
 * context's beta at beta_target.  Needs 0 < factor < 1, beta_start > 0. */
int claire_solve_continuation(claire_ctx *ctx, float *v_inout, double beta_target,
                              double beta_start, double factor, const claire_solve_opts *opts,
                              claire_solve_report *report, int *levels);

/* ---- instrumentation -------------------------------------------------- */

/* Kernel classes timed by the profiler (CLAIRE_K_DERIV: spectral first
 * derivatives by axis transforms, three passes per gradient or divergence). */
enum {
    CLAIRE_K_FOOTPOINT = 0, CLAIRE_K_STATE = 1, CLAIRE_K_ADJOINT = 2,
    CLAIRE_K_INCSTATE = 3, CLAIRE_K_INCADJ = 4, CLAIRE_K_BODYFORCE = 5,
    CLAIRE_K_FFT_R2C = 6, CLAIRE_K_FFT_C2C = 7, CLAIRE_K_FFT_MUL = 8,
    CLAIRE_K_FFT_C2R = 9, CLAIRE_K_REDUCE = 10, CLAIRE_K_VECTOR = 11,
    CLAIRE_K_INTERP = 12, CLAIRE_K_FD = 13, CLAIRE_K_DERIV = 14, CLAIRE_K_COUNT = 15
};

/* Enable (1) or disable (0) per-launch CUDA-event timing of every kernel the
 * context launches (on its stream); enabling clears earlier records. */
int claire_profile_enable(claire_ctx *ctx, int on);

/* For one kernel class, since profiling was enabled: the number of timed
 * launch groups, their summed device time (ms) and their summed algorithmic
 * HBM bytes (every field a launch reads or writes counted once; a gathered
 * field counted as one read).  Any output pointer may be NULL.  Synchronizes. */
int claire_profile_read(claire_ctx *ctx, int kernel_class, long *launches, double *total_ms,
                        double *total_bytes);

/* Total number of kernels the context has launched since creation. */
int claire_launch_count(const claire_ctx *ctx, long *launches);

/* Device bytes held by the context. */
int claire_workspace_bytes(const claire_ctx *ctx, size_t *bytes);

/* Cap, for every context of the process, on the device bytes one context may
 * allocate (its workspace at claire_create and buffers it allocates later,
 * e.g. the checkpoints of the differentiable form); 0 (the default) removes
 * the cap.  An allocation that would pass the cap fails with CLAIRE_ERR_OOM
 * before cudaMalloc is called, exactly as a failed cudaMalloc does: the
 * context (or claire_create) reports the error and stays usable.  For
 * callers that budget device memory, and to test the out-of-memory paths
 * without exhausting the device.  Contexts created earlier keep what they
 * hold.  No counterpart in the paper. */
int claire_set_workspace_limit(size_t bytes);

/* ---- preconditioner without device allocation --------------------------
 * The paper has no counterpart of this entry point; it exists for callers
 * that cannot allocate device memory (a host framework that owns the whole
 * device heap, code that may not call cudaMalloc/cudaFree because they
 * synchronize, a fixed memory budget).  It computes the same
 * s = (beta*A)^{-1} r as claire_precond for an nx*ny*nz grid without a
 * context, on `stream` (a cudaStream_t; NULL = legacy), and allocates
 * nothing: its scratch (FFT half spectra and twiddle tables) is a file-scope
 * device array of fixed size that every GPU loading the library holds until
 * exit.  Limit: 3 * nx * ny * p3 <= 442368 complex values, p3 = (nz/2 + 1)
 * rounded up to a multiple of 4 (a 64^3 grid fits); larger grids, invalid
 * sizes, beta <= 0, gamma < 0 or NULL pointers return CLAIRE_ERR_ARG with a
 * message in claire_last_error(NULL).  r and s are device float[3][N] and
 * may be equal.  The first call on each device looks up the array's device
 * address (so make it before any stream capture) and keeps it for the life of
 * the process: a device reset (cudaDeviceReset) after that first call is not
 * supported by this entry point.  All calls on a device share
 * the array: calls that overlap on the GPU race and must be serialized by the
 * caller.  Returns as soon as the work is enqueued. */
int claire_precond_noalloc(int nx, int ny, int nz, double beta, double gamma, const float *r,
                           float *s, void *stream);

/* Debug build only (compiled with -DCLAIRE_CHECKS, libclaire_gb_checks.so):
 * the number of shared-memory box stencils the transport kernels found
 * outside the part of the box their copy wrote since the last reset (each is
 * counted and not read).  Synchronizes the device; reset != 0 clears the
 * count.  The release build returns CLAIRE_ERR_STATE with *count = 0.  No
 * counterpart in the paper (its kernels are checked on the CPU here too). */
int claire_check_count(unsigned long long *count, int reset);

/* Message of the last error on ctx (or of the last failed claire_create when
 * ctx is NULL); never NULL. */
const char *claire_last_error(const claire_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* CLAIRE_H */
