"""Thin ctypes binding of the C ABI in ``include/claire.h``.

Argument marshalling only: every step of the registration runs in the CUDA
kernels of ``libclaire_gb.so``.  Fields are torch CUDA tensors (float32,
contiguous; vectors shaped ``[3, nx, ny, nz]``) whose device pointers are
passed through.  There is no CPU path: if the library is missing or no GPU is
present the calls raise.

The function names mirror the C entry points (``claire_create``,
``claire_gradient``, ...); :class:`Registration` bundles them for convenience.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libclaire_gb.so")

CLAIRE_OK = 0
STATUS = {0: "CLAIRE_OK", 1: "CLAIRE_ERR_ARG", 2: "CLAIRE_ERR_OOM", 3: "CLAIRE_ERR_CUDA",
          4: "CLAIRE_ERR_STATE", 5: "CLAIRE_ERR_NONFINITE", 6: "CLAIRE_ERR_LINESEARCH",
          7: "CLAIRE_ERR_PCG_BREAKDOWN", 8: "CLAIRE_ERR_TIMEOUT"}

FIELD = dict(dispm=0, dispp=1, state=2, gradm=3, divv=4, adjf=5, adj=6, incadj=7, incst=8)
KERNEL = dict(footpoint=0, state=1, adjoint=2, incstate=3, incadj=4, bodyforce=5, fft_r2c=6,
              fft_c2c=7, fft_mul=8, fft_c2r=9, reduce=10, vector=11, interp=12, fd=13, deriv=14)

EXPORTED = [
    "claire_create", "claire_create_ex", "claire_destroy", "claire_set_stream", "claire_set_params",
    "claire_set_images", "claire_forward", "claire_objective", "claire_linearize",
    "claire_gradient", "claire_hess_matvec", "claire_precond", "claire_grad", "claire_div",
    "claire_apply_A", "claire_interp", "claire_get_field", "claire_solve_opts_default",
    "claire_solve", "claire_profile_enable", "claire_profile_read", "claire_launch_count",
    "claire_workspace_bytes", "claire_last_error", "claire_precond_noalloc",
    "claire_precond_h0", "claire_solve_continuation", "claire_set_discretization", "claire_solve_batch",
    "claire_mismatch_forward", "claire_mismatch_backward", "claire_solve_host", "claire_set_workspace_limit",
    "claire_checkpoint_stride", "claire_check_count",
]


class ClaireError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class SolveOpts(ctypes.Structure):
    _fields_ = [("max_gn", ctypes.c_int), ("max_pcg", ctypes.c_int), ("fixed_pcg", ctypes.c_int),
                ("eps_n", ctypes.c_double), ("armijo_c1", ctypes.c_double),
                ("max_ls", ctypes.c_int), ("precond", ctypes.c_int), ("eps_h0", ctypes.c_double),
                ("max_inner", ctypes.c_int)]


class SolveReport(ctypes.Structure):
    _fields_ = [("n_gn", ctypes.c_int), ("n_pcg", ctypes.c_int), ("n_matvec", ctypes.c_int),
                ("n_precond", ctypes.c_int), ("n_ls", ctypes.c_int), ("status", ctypes.c_int),
                ("J0", ctypes.c_double), ("J", ctypes.c_double), ("g0", ctypes.c_double),
                ("g", ctypes.c_double), ("grel", ctypes.c_double),
                ("mismatch_rel", ctypes.c_double), ("n_inner", ctypes.c_long),
                ("t_grad_ms", ctypes.c_double),
                ("t_hess_ms", ctypes.c_double), ("t_pc_ms", ctypes.c_double),
                ("t_obj_ms", ctypes.c_double), ("t_pcg_ms", ctypes.c_double),
                ("t_total_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load(path: str = LIB_PATH):
    """Load libclaire_gb.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    L = ctypes.CDLL(path)
    P, I, D, V = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    pd = ctypes.POINTER(ctypes.c_double)
    sig = {
        "claire_create": [I, I, I, I, D, D, ctypes.POINTER(P)],
        "claire_create_ex": [I, I, I, I, D, D, I, ctypes.POINTER(P)],
        "claire_destroy": [P], "claire_set_stream": [P, V], "claire_set_params": [P, D, D],
        "claire_set_images": [P, V, V], "claire_forward": [P, V, V, pd],
        "claire_objective": [P, V, pd, pd], "claire_linearize": [P, V],
        "claire_gradient": [P, V, V, pd], "claire_hess_matvec": [P, V, V, V],
        "claire_precond": [P, V, V], "claire_grad": [P, V, V], "claire_div": [P, V, V],
        "claire_apply_A": [P, V, V], "claire_interp": [P, V, V, V],
        "claire_get_field": [P, I, I, V],
        "claire_solve": [P, V, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveReport)],
        "claire_solve_host": [P, V, V, V, V, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveReport)],
        "claire_solve_batch": [ctypes.POINTER(P), ctypes.POINTER(V), I, ctypes.POINTER(SolveOpts),
                               ctypes.POINTER(SolveReport)],
        "claire_profile_enable": [P, I],
        "claire_profile_read": [P, I, ctypes.POINTER(ctypes.c_long), pd, pd],
        "claire_launch_count": [P, ctypes.POINTER(ctypes.c_long)],
        "claire_workspace_bytes": [P, ctypes.POINTER(ctypes.c_size_t)],
        "claire_set_workspace_limit": [ctypes.c_size_t],
        "claire_precond_noalloc": [I, I, I, D, D, V, V, V],
        "claire_precond_h0": [P, V, V, D, I, I, ctypes.POINTER(ctypes.c_int)],
        "claire_set_discretization": [P, I, I],
        "claire_mismatch_forward": [P, V, V, pd, I],
        "claire_mismatch_backward": [P, D, V, V],
        "claire_checkpoint_stride": [P, ctypes.POINTER(ctypes.c_int)],
        "claire_check_count": [ctypes.POINTER(ctypes.c_ulonglong), I],
        "claire_solve_continuation": [P, V, D, D, D, ctypes.POINTER(SolveOpts),
                                      ctypes.POINTER(SolveReport), ctypes.POINTER(ctypes.c_int)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.claire_solve_opts_default.argtypes = [ctypes.POINTER(SolveOpts)]
    L.claire_solve_opts_default.restype = None
    L.claire_last_error.argtypes = [P]
    L.claire_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _ptr(t, shape=None, name="field"):
    """Device pointer of a contiguous float32 CUDA tensor.  With ``shape``, the
    tensor's shape must equal it: the C side reads and writes exactly that many
    floats through the pointer, so a wrong shape is rejected here, before any
    pointer crosses into the library."""
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(t.shape)}, expected {tuple(shape)}")
    if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{name}: fields must be contiguous float32 CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(t):
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError("host fields must be contiguous float32 CPU tensors (page-locked for overlap)")
    return ctypes.c_void_p(t.data_ptr())


def _check(ctx, rc):
    if rc != CLAIRE_OK:
        msg = load().claire_last_error(ctx).decode()
        raise ClaireError(rc, msg)


@dataclass
class Report:
    n_gn: int
    n_pcg: int
    n_matvec: int
    n_precond: int
    n_ls: int
    status: int
    J0: float
    J: float
    g0: float
    g: float
    grel: float
    mismatch_rel: float
    n_inner: int
    t_grad_ms: float
    t_hess_ms: float
    t_pc_ms: float
    t_obj_ms: float
    t_pcg_ms: float
    t_total_ms: float


def set_workspace_limit(nbytes):
    """Cap the device bytes any one context may allocate (0: no cap); an
    allocation past it fails with CLAIRE_ERR_OOM (claire_set_workspace_limit)."""
    rc = load().claire_set_workspace_limit(int(nbytes))
    if rc != CLAIRE_OK:
        raise ClaireError(rc, "claire_set_workspace_limit")


def check_count(reset=False):
    """Box-stencil violations counted by the debug build (claire_check_count);
    raises in the release build, which has no counter."""
    n = ctypes.c_ulonglong(0)
    rc = load().claire_check_count(ctypes.byref(n), 1 if reset else 0)
    if rc != CLAIRE_OK:
        raise ClaireError(rc, "claire_check_count: the loaded library is not the checks build")
    return n.value


def precond_noalloc(r, s, beta, gamma, stream=None):
    """s = (beta*A)^{-1} r through claire_precond_noalloc (no device allocation
    inside the library); r, s: float32 CUDA tensors [3, nx, ny, nz]."""
    if not isinstance(r, torch.Tensor) or r.dim() != 4 or r.shape[0] != 3:
        raise ValueError("precond_noalloc: r must be a [3, nx, ny, nz] tensor")
    shape = tuple(r.shape)
    pr, ps = _ptr(r, shape, "r"), _ptr(s, shape, "s")
    L = load()
    st = stream if stream is not None else torch.cuda.current_stream()
    nx, ny, nz = (int(x) for x in shape[1:])
    rc = L.claire_precond_noalloc(nx, ny, nz, float(beta), float(gamma), pr, ps,
                                  ctypes.c_void_p(st.cuda_stream))
    if rc != CLAIRE_OK:
        raise ClaireError(rc, L.claire_last_error(None).decode())
    return s


def solve_batch(regs, vs, check=True, **opts):
    """Solve the registrations ``regs`` (Registration objects, distinct) with
    velocities ``vs`` (float32 CUDA tensors, in/out) together through
    claire_solve_batch: up to eight host threads with a CUDA stream each take
    the pairs largest grid first; results bitwise those of ``reg.solve(v)``
    one by one.  Returns the reports."""
    n = len(regs)
    if n != len(vs) or n == 0:
        raise ValueError("need as many velocities as registrations (>= 1)")
    if isinstance(opts.get("precond"), str):
        opts["precond"] = Registration.PRECOND[opts["precond"]]
    o = Registration.default_opts(**opts)
    ptrs = [r._vec(v, "v") for r, v in zip(regs, vs)]
    hs = (ctypes.c_void_p * n)(*[r.handle for r in regs])
    ps = (ctypes.c_void_p * n)(*ptrs)
    reps = (SolveReport * n)()
    rc = load().claire_solve_batch(hs, ps, n, ctypes.byref(o), reps)
    if check and rc != CLAIRE_OK:
        bad = [i for i in range(n) if reps[i].status != CLAIRE_OK]
        if bad:
            _check(regs[bad[0]].handle, rc)
        raise ClaireError(rc, load().claire_last_error(None).decode())
    return [Report(**reps[i].as_dict()) for i in range(n)]


class Registration:
    """One registration problem on an nx*ny*nz grid (a claire_ctx).

    All field arguments are torch CUDA tensors on the current device; the
    context runs on torch's current stream unless ``stream`` is given."""

    PRECISION = {"fp32": 0, "fp16": 1}

    def __init__(self, shape, nt, beta, gamma, stream=None, precision="fp32"):
        """precision: "fp32" (the paper's setting) or "fp16" (stored state,
        state gradient and adjoint trajectories in FP16, FP32 arithmetic)."""
        L = load()
        h = ctypes.c_void_p()
        nx, ny, nz = (int(s) for s in shape)
        prec = self.PRECISION[precision] if isinstance(precision, str) else int(precision)
        rc = L.claire_create_ex(nx, ny, nz, int(nt), float(beta), float(gamma), prec, ctypes.byref(h))
        if rc != CLAIRE_OK:
            raise ClaireError(rc, L.claire_last_error(None).decode())
        self._h = h
        self.shape = (nx, ny, nz)
        self.nt, self.beta, self.gamma = nt, beta, gamma
        self.precision = precision
        st = stream if stream is not None else torch.cuda.current_stream()
        self._stream = st
        _check(h, L.claire_set_stream(h, ctypes.c_void_p(st.cuda_stream)))

    # ---- lifetime ----
    def close(self):
        if getattr(self, "_h", None):
            load().claire_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    def _c(self, name, *args):
        _check(self._h, getattr(load(), name)(self._h, *args))

    def _new(self, *lead):
        return torch.empty(lead + self.shape, device="cuda", dtype=torch.float32)

    def _vec(self, t, name="vector field"):
        """pointer of a [3, nx, ny, nz] field of this grid (None passes)"""
        return _ptr(t, (3,) + self.shape, name)

    def _scal(self, t, name="scalar field"):
        """pointer of an [nx, ny, nz] field of this grid (None passes)"""
        return _ptr(t, self.shape, name)

    # ---- API ----
    def set_params(self, beta, gamma):
        self._c("claire_set_params", float(beta), float(gamma))
        self.beta, self.gamma = beta, gamma

    def set_discretization(self, interp="cubic", deriv="spectral"):
        """interp "cubic" | "linear"; deriv "spectral" | "fd8" (Sections 4.1, 4.2)."""
        self._c("claire_set_discretization", 1 if interp == "linear" else 3,
                1 if deriv == "fd8" else 0)

    def set_images(self, m0, m1):
        self._c("claire_set_images", self._scal(m0, "m0"), self._scal(m1, "m1"))

    def forward(self, v, want_mismatch=True):
        pv = self._vec(v, "v")
        m = self._new()
        mis = ctypes.c_double(0)
        self._c("claire_forward", pv, self._scal(m, "m"), ctypes.byref(mis) if want_mismatch else None)
        return m, mis.value

    def mismatch_forward(self, v, checkpoint_stride=2, m_final=None):
        """(m(1), mismatch) keeping the state every checkpoint_stride steps
        (0: chosen from the free device memory, see checkpoint_stride())."""
        pv = self._vec(v, "v")
        m = m_final if m_final is not None else self._new()
        mis = ctypes.c_double(0)
        self._c("claire_mismatch_forward", pv, self._scal(m, "m_final"), ctypes.byref(mis),
                int(checkpoint_stride))
        return m, mis.value

    def mismatch_backward(self, grad_mismatch, grad_m_final=None, out=None):
        """Euclidean gradient w.r.t. v of grad_mismatch * mismatch +
        <grad_m_final, m(1)> at the last mismatch_forward."""
        pg = self._scal(grad_m_final, "grad_m_final")
        g = out if out is not None else self._new(3)
        self._c("claire_mismatch_backward", float(grad_mismatch), pg, self._vec(g, "out"))
        return g

    def checkpoint_stride(self):
        """stride of the differentiable form (0 before its first forward)"""
        k = ctypes.c_int(0)
        self._c("claire_checkpoint_stride", ctypes.byref(k))
        return k.value

    def objective(self, v):
        J, mis = ctypes.c_double(0), ctypes.c_double(0)
        self._c("claire_objective", self._vec(v, "v"), ctypes.byref(J), ctypes.byref(mis))
        return J.value, mis.value

    def linearize(self, v):
        self._c("claire_linearize", self._vec(v, "v"))

    def gradient(self, v, out=None, want_objective=True):
        pv = self._vec(v, "v")
        g = out if out is not None else self._new(3)
        J = ctypes.c_double(0)
        self._c("claire_gradient", pv, self._vec(g, "out"), ctypes.byref(J) if want_objective else None)
        return g, J.value

    def hess_matvec(self, v, vt, out=None):
        pv, pvt = self._vec(v, "v"), self._vec(vt, "vt")
        Hv = out if out is not None else self._new(3)
        self._c("claire_hess_matvec", pv, pvt, self._vec(Hv, "out"))
        return Hv

    def precond(self, r, out=None):
        pr = self._vec(r, "r")
        s = out if out is not None else self._new(3)
        self._c("claire_precond", pr, self._vec(s, "out"))
        return s

    def precond_h0(self, r, out=None, tol=1e-3, maxit=500, two_level=False):
        """InvH0 or its two-level variant: (s, inner iterations) with
        s = H0^{-1} r at the cached linearization."""
        pr = self._vec(r, "r")
        s = out if out is not None else self._new(3)
        it = ctypes.c_int(0)
        self._c("claire_precond_h0", pr, self._vec(s, "out"), float(tol), int(maxit), int(bool(two_level)),
                ctypes.byref(it))
        return s, it.value

    def grad(self, f):
        pf = self._scal(f, "f")
        g = self._new(3)
        self._c("claire_grad", pf, self._vec(g))
        return g

    def div(self, v):
        pv = self._vec(v, "v")
        d = self._new()
        self._c("claire_div", pv, self._scal(d))
        return d

    def apply_A(self, v):
        pv = self._vec(v, "v")
        out = self._new(3)
        self._c("claire_apply_A", pv, self._vec(out))
        return out

    def interp(self, f, disp):
        pf, pd = self._scal(f, "f"), self._vec(disp, "disp")
        out = self._new()
        self._c("claire_interp", pf, pd, self._scal(out))
        return out

    def field(self, name, j=0):
        comps = 3 if name in ("dispm", "dispp", "gradm") else 1
        out = self._new(3) if comps == 3 else self._new()
        self._c("claire_get_field", FIELD[name], int(j), _ptr(out))
        return out

    @staticmethod
    def default_opts(**kw):
        o = SolveOpts()
        load().claire_solve_opts_default(ctypes.byref(o))
        for k, val in kw.items():
            setattr(o, k, val)
        return o

    PRECOND = {"invA": 0, "invH0": 1, "2LinvH0": 2}

    def solve(self, v_inout, check=True, **opts):
        """opts: max_gn, max_pcg, fixed_pcg, eps_n, armijo_c1, max_ls,
        precond ("invA" | "invH0" | "2LinvH0" or the enum value), eps_h0, max_inner."""
        pv = self._vec(v_inout, "v")
        if isinstance(opts.get("precond"), str):
            opts["precond"] = self.PRECOND[opts["precond"]]
        o = self.default_opts(**opts)
        rep = SolveReport()
        rc = load().claire_solve(self._h, pv, ctypes.byref(o), ctypes.byref(rep))
        if check and rc not in (CLAIRE_OK,):
            _check(self._h, rc)
        return Report(**rep.as_dict())

    def solve_host(self, m0, m1, v_in, v_out=None, check=True, **opts):
        """set_images + solve with host (CPU) tensors, the copies overlapped
        with the computation (pin the tensors for the overlap); the result
        lands in v_out (default: v_in) before the call returns."""
        if v_out is None:
            v_out = v_in
        for t, want, nm in ((m0, self.shape, "m0"), (m1, self.shape, "m1"), (v_in, (3,) + self.shape, "v_in"),
                            (v_out, (3,) + self.shape, "v_out")):
            if not isinstance(t, torch.Tensor) or tuple(t.shape) != want:
                raise ValueError(f"solve_host: {nm} must have shape {want}")
        if isinstance(opts.get("precond"), str):
            opts["precond"] = self.PRECOND[opts["precond"]]
        o = self.default_opts(**opts)
        rep = SolveReport()
        rc = load().claire_solve_host(self._h, _host_ptr(m0), _host_ptr(m1), _host_ptr(v_in), _host_ptr(v_out),
                                      ctypes.byref(o), ctypes.byref(rep))
        if check and rc not in (CLAIRE_OK,):
            _check(self._h, rc)
        return Report(**rep.as_dict())

    def solve_continuation(self, v_inout, beta_target, beta_start=1.0, factor=0.1, check=True,
                           **opts):
        """beta-continuation (InvA while beta > 0.5, opts["precond"] below);
        returns (report, levels).  The context's beta ends at beta_target."""
        if isinstance(opts.get("precond"), str):
            opts["precond"] = self.PRECOND[opts["precond"]]
        o = self.default_opts(**opts)
        rep = SolveReport()
        lev = ctypes.c_int(0)
        rc = load().claire_solve_continuation(self._h, self._vec(v_inout, "v"), float(beta_target),
                                              float(beta_start), float(factor), ctypes.byref(o),
                                              ctypes.byref(rep), ctypes.byref(lev))
        if check and rc != CLAIRE_OK:
            _check(self._h, rc)
        self.beta = beta_target
        return Report(**rep.as_dict()), lev.value

    def profile_enable(self, on=True):
        self._c("claire_profile_enable", 1 if on else 0)

    def profile_read(self, kernel):
        """(launch groups, device ms, algorithmic bytes) of one kernel class."""
        n, ms, by = ctypes.c_long(0), ctypes.c_double(0), ctypes.c_double(0)
        self._c("claire_profile_read", KERNEL[kernel] if isinstance(kernel, str) else int(kernel),
                ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by))
        return n.value, ms.value, by.value

    def launch_count(self):
        n = ctypes.c_long(0)
        _check(self._h, load().claire_launch_count(self._h, ctypes.byref(n)))
        return n.value

    def workspace_bytes(self):
        n = ctypes.c_size_t(0)
        _check(self._h, load().claire_workspace_bytes(self._h, ctypes.byref(n)))
        return n.value
