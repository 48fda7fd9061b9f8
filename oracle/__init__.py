"""FP64 CPU oracle for the GN-Krylov registration method (arXiv 2008.12820).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only users.  The CUDA library never
calls it and shares no code with it.

The arithmetic lives in ``claire_oracle.c`` (plain C, IEEE double, OpenMP over
independent grid points).  This module compiles it with gcc on first use and
wraps each entry point for numpy arrays.  Every wrapped function cites the part
of the paper it follows in the C source.

Field layout: scalar fields ``[N1, N2, N3]`` (x3 contiguous); vector fields
``[3, N1, N2, N3]``; velocities in domain units on Omega = [0, 2*pi)^3.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "claire_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.c_int
_L = ctypes.c_long


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (-O2, OpenMP, no fast-math)."""
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class _SolveOpts(ctypes.Structure):
    _fields_ = [("max_gn", _I), ("max_pcg", _I), ("fixed_pcg", _I), ("eps_n", ctypes.c_double),
                ("armijo_c1", ctypes.c_double), ("max_ls", _I), ("pc", _I),
                ("eps_h0", ctypes.c_double), ("max_inner", _I)]


class _SolveReport(ctypes.Structure):
    _fields_ = [("n_gn", _I), ("n_pcg", _I), ("n_matvec", _I), ("n_precond", _I), ("status", _I),
                ("J0", ctypes.c_double), ("J", ctypes.c_double), ("g0", ctypes.c_double),
                ("g", ctypes.c_double), ("grel", ctypes.c_double),
                ("mismatch_rel", ctypes.c_double), ("n_inner", _L)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.or_fft3.argtypes = [_I, _I, _I, _D, _I]
        L.or_grad.argtypes = [_I, _I, _I, _D, _D]
        L.or_div.argtypes = [_I, _I, _I, _D, _D]
        L.or_apply_A.argtypes = [_I, _I, _I, ctypes.c_double, ctypes.c_double, _D, _D]
        L.or_apply_Ainv.argtypes = [_I, _I, _I, ctypes.c_double, ctypes.c_double, _D, _D]
        L.or_lagrange.argtypes = [_I, ctypes.c_double]
        L.or_lagrange.restype = ctypes.c_double
        L.or_interp.argtypes = [_I, _I, _I, _D, _L, _D, _D, _D, _D]
        L.or_footpoints.argtypes = [_I, _I, _I, _I, _D, _I, _D]
        L.or_state.argtypes = [_I, _I, _I, _I, _D, _D, _D]
        L.or_adjoint.argtypes = [_I, _I, _I, _I, _D, _D, _D, _D, _D]
        L.or_incstate.argtypes = [_I, _I, _I, _I, _D, _D, _D, _D]
        L.or_bodyforce.argtypes = [_L, _I, _D, _D, _D]
        L.or_create.argtypes = [_I, _I, _I, _I, ctypes.c_double, ctypes.c_double, _D, _D]
        L.or_create.restype = ctypes.c_void_p
        L.or_destroy.argtypes = [ctypes.c_void_p]
        L.or_linearize.argtypes = [ctypes.c_void_p, _D]
        for name in ("or_state_ptr", "or_gradstate_ptr", "or_dispm_ptr", "or_dispp_ptr",
                     "or_div_ptr", "or_divp_ptr"):
            getattr(L, name).argtypes = [ctypes.c_void_p]
            getattr(L, name).restype = _D
        L.or_objective.argtypes = [ctypes.c_void_p, _D, _D, _D, _D]
        L.or_objective.restype = ctypes.c_double
        L.or_gradient.argtypes = [ctypes.c_void_p, _D, _D, _D, _D]
        L.or_matvec.argtypes = [ctypes.c_void_p, _D, _D, _D, _D]
        L.or_matvec.restype = _I
        L.or_precond.argtypes = [ctypes.c_void_p, _D, _D]
        L.or_pcg_dense.argtypes = [_L, _D, _D, _D, _D, ctypes.c_double, _L, _I,
                                   ctypes.POINTER(_I), _D]
        L.or_pcg_dense.restype = _L
        L.or_solve.argtypes = [ctypes.c_void_p, _D, ctypes.POINTER(_SolveOpts),
                               ctypes.POINTER(_SolveReport)]
        L.or_solve.restype = _I
        L.or_det_grad_y.argtypes = [_I, _I, _I, _I, _D, _D]
        L.or_h0_matvec.argtypes = [_I, _I, _I, ctypes.c_double, ctypes.c_double, _D, _D, _D]
        L.or_invh0.argtypes = [_I, _I, _I, ctypes.c_double, ctypes.c_double, _D, _D, _D,
                               ctypes.c_double, _L]
        L.or_invh0.restype = _L
        L.or_invh0_2l.argtypes = L.or_invh0.argtypes
        L.or_invh0_2l.restype = _L
        _I3 = _I * 3
        L.or_restrict.argtypes = [_I3, _I3, _D, _D]
        L.or_prolong.argtypes = [_I3, _I3, _D, _D]
        L.or_highpass.argtypes = [_I3, _I3, _D, _D]
        L.or_set_discretization.argtypes = [ctypes.c_void_p, _I, _I]
        L.or_grad_fd8.argtypes = [_I, _I, _I, _D, _D]
        L.or_div_fd8.argtypes = [_I, _I, _I, _D, _D]
        L.or_lerp.argtypes = [_I, _I, _I, _D, _L, _D, _D, _D, _D]
        L.or_solve_continuation.argtypes = [ctypes.c_void_p, _D, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, ctypes.POINTER(_SolveOpts),
                                            ctypes.POINTER(_SolveReport), ctypes.POINTER(_I)]
        L.or_solve_continuation.restype = _I
        _lib = L
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _shape(f) -> tuple:
    s = tuple(int(x) for x in np.shape(f))
    return s[-3:]


# --------------------------------------------------------------------------
# primitives (each wraps one C function)
# --------------------------------------------------------------------------

def fft3(a: np.ndarray, sign: int = -1) -> np.ndarray:
    """Unnormalized 3D DFT, sign -1 forward / +1 backward (own mixed-radix FFT)."""
    z = np.ascontiguousarray(a, dtype=np.complex128).copy()
    n1, n2, n3 = z.shape
    lib().or_fft3(n1, n2, n3, z.ctypes.data_as(_D), sign)
    return z


def grad(f: np.ndarray) -> np.ndarray:
    f = _f64(f)
    out = np.empty((3,) + f.shape)
    lib().or_grad(*f.shape, _p(f), _p(out))
    return out


def div(v: np.ndarray) -> np.ndarray:
    v = _f64(v)
    out = np.empty(v.shape[1:])
    lib().or_div(*v.shape[1:], _p(v), _p(out))
    return out


def apply_A(v: np.ndarray, beta: float, gamma: float) -> np.ndarray:
    """beta*A v with beta*A = -beta*Laplace - gamma*grad div (spectral)."""
    v = _f64(v)
    out = np.empty_like(v)
    lib().or_apply_A(*v.shape[1:], beta, gamma, _p(v), _p(out))
    return out


def apply_Ainv(v: np.ndarray, beta: float, gamma: float) -> np.ndarray:
    """(beta*A)^{-1} v, identity on the zero wavenumber."""
    v = _f64(v)
    out = np.empty_like(v)
    lib().or_apply_Ainv(*v.shape[1:], beta, gamma, _p(v), _p(out))
    return out


def grad_fd8(f: np.ndarray) -> np.ndarray:
    """Eighth-order central-difference gradient (Section 4.2)."""
    f = _f64(f)
    out = np.empty((3,) + f.shape)
    lib().or_grad_fd8(*f.shape, _p(f), _p(out))
    return out


def div_fd8(v: np.ndarray) -> np.ndarray:
    v = _f64(v)
    out = np.empty(v.shape[1:])
    lib().or_div_fd8(*v.shape[1:], _p(v), _p(out))
    return out


def lerp(f: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Periodic trilinear interpolation of f at points q[3, ...] (index units)."""
    f = _f64(f)
    q = _f64(q).reshape(3, -1)
    q1, q2, q3 = (np.ascontiguousarray(q[d]) for d in range(3))
    out = np.empty(q.shape[1])
    lib().or_lerp(*f.shape, _p(f), q.shape[1], _p(q1), _p(q2), _p(q3), _p(out))
    return out


def lagrange(a: int, t: float) -> float:
    return lib().or_lagrange(a, t)


def interp(f: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Periodic cubic Lagrange interpolation of f at points q[3, ...] (index units)."""
    f = _f64(f)
    q = _f64(q).reshape(3, -1)
    q1, q2, q3 = (np.ascontiguousarray(q[d]) for d in range(3))
    out = np.empty(q.shape[1])
    lib().or_interp(*f.shape, _p(f), q.shape[1], _p(q1), _p(q2), _p(q3), _p(out))
    return out


def footpoints(v: np.ndarray, nt: int, sign: int) -> np.ndarray:
    """RK2 (Heun) foot point displacement in index units; sign -1: X-, +1: X+."""
    v = _f64(v)
    out = np.empty_like(v)
    lib().or_footpoints(*v.shape[1:], nt, _p(v), sign, _p(out))
    return out


def state(dispm: np.ndarray, m0: np.ndarray, nt: int) -> np.ndarray:
    dispm, m0 = _f64(dispm), _f64(m0)
    out = np.empty((nt + 1,) + m0.shape)
    lib().or_state(*m0.shape, nt, _p(dispm), _p(m0), _p(out))
    return out


def adjoint(dispp, d, dp, lfinal, nt: int) -> np.ndarray:
    dispp, d, dp, lfinal = _f64(dispp), _f64(d), _f64(dp), _f64(lfinal)
    out = np.empty((nt + 1,) + lfinal.shape)
    lib().or_adjoint(*lfinal.shape, nt, _p(dispp), _p(d), _p(dp), _p(lfinal), _p(out))
    return out


def incstate(dispm, gmhist, vt, nt: int) -> np.ndarray:
    dispm, gmhist, vt = _f64(dispm), _f64(gmhist), _f64(vt)
    out = np.empty((nt + 1,) + vt.shape[1:])
    lib().or_incstate(*vt.shape[1:], nt, _p(dispm), _p(gmhist), _p(vt), _p(out))
    return out


def bodyforce(lhist, gmhist) -> np.ndarray:
    lhist, gmhist = _f64(lhist), _f64(gmhist)
    nt = lhist.shape[0] - 1
    N = int(np.prod(lhist.shape[1:]))
    out = np.empty((3,) + lhist.shape[1:])
    lib().or_bodyforce(N, nt, _p(lhist), _p(gmhist), _p(out))
    return out


def det_grad_y(v: np.ndarray, nt: int) -> np.ndarray:
    v = _f64(v)
    out = np.empty(v.shape[1:])
    lib().or_det_grad_y(*v.shape[1:], nt, _p(v), _p(out))
    return out


def h0_matvec(s, gm, beta0, gamma):
    """H0 s = beta0 A s + grad m (grad m . s) (zero-velocity Hessian)."""
    s, gm = _f64(s), _f64(gm)
    out = np.empty_like(s)
    lib().or_h0_matvec(*s.shape[1:], beta0, gamma, _p(gm), _p(s), _p(out))
    return out


def invh0(r, gm, beta0, gamma, tol, maxit=500, two_level=False):
    """PCG solve of H0 s = r, preconditioned by (beta0 A)^{-1}; two_level solves
    on the half grid and adds the high-pass part (Algorithm 2)."""
    r, gm = _f64(r), _f64(gm)
    out = np.empty_like(r)
    f = lib().or_invh0_2l if two_level else lib().or_invh0
    it = f(*r.shape[1:], beta0, gamma, _p(gm), _p(r), _p(out), tol, maxit)
    return out, int(it)


def _resample(fn, f, shape_out):
    f = _f64(f)
    out = np.empty(shape_out)
    n_in = (ctypes.c_int * 3)(*f.shape)
    n_out = (ctypes.c_int * 3)(*shape_out)
    fn(n_in, n_out, _p(f), _p(out))
    return out


def restrict(f, shape_c):
    """Spectral restriction to a coarser grid (|k_d| < nc_d/2 kept)."""
    return _resample(lib().or_restrict, f, tuple(shape_c))


def prolong(fc, shape_f):
    """Spectral prolongation (zero padding of the coarse band)."""
    fc = _f64(fc)
    out = np.empty(tuple(shape_f))
    lib().or_prolong((ctypes.c_int * 3)(*fc.shape), (ctypes.c_int * 3)(*shape_f), _p(fc), _p(out))
    return out


def highpass(f, shape_c):
    f = _f64(f)
    out = np.empty_like(f)
    lib().or_highpass((ctypes.c_int * 3)(*f.shape), (ctypes.c_int * 3)(*shape_c), _p(f), _p(out))
    return out


def pcg_dense(H: np.ndarray, P: np.ndarray, b: np.ndarray, tol: float, maxit: int,
              fixed: bool = False):
    """Run the oracle's PCG routine on dense matrices (for checking PCG itself)."""
    H, P, b = _f64(H), _f64(P), _f64(b)
    n = b.shape[0]
    x = np.empty(n)
    flag = _I(0)
    rel = ctypes.c_double(0)
    it = lib().or_pcg_dense(n, _p(H), _p(P), _p(b), _p(x), tol, maxit, int(fixed),
                            ctypes.byref(flag), ctypes.byref(rel))
    return x, int(it), int(flag.value), float(rel.value)


# --------------------------------------------------------------------------
# problem object
# --------------------------------------------------------------------------

@dataclass
class SolveReport:
    n_gn: int
    n_pcg: int
    n_matvec: int
    n_precond: int
    status: int
    J0: float
    J: float
    g0: float
    g: float
    grel: float
    mismatch_rel: float
    n_inner: int


class Problem:
    """Images m0, m1 and parameters (nt, beta, gamma) on an N1 x N2 x N3 grid."""

    def __init__(self, m0, m1, nt: int, beta: float, gamma: float):
        m0, m1 = _f64(m0), _f64(m1)
        self.shape = m0.shape
        self.N = int(np.prod(self.shape))
        self.nt, self.beta, self.gamma = nt, beta, gamma
        self._h = lib().or_create(*self.shape, nt, beta, gamma, _p(m0), _p(m1))

    def set_discretization(self, interp="cubic", deriv="spectral"):
        """interp: "cubic" | "linear"; deriv: "spectral" | "fd8" (Sections 4.1, 4.2)."""
        lib().or_set_discretization(self._h, 1 if interp == "linear" else 3,
                                    1 if deriv == "fd8" else 0)

    def close(self):
        if self._h:
            lib().or_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _view(self, fn, shape):
        ptr = getattr(lib(), fn)(self._h)
        return np.ctypeslib.as_array(ptr, shape=shape).copy()

    def linearize(self, v):
        v = _f64(v)
        lib().or_linearize(self._h, _p(v))

    # views of the stored linearization (copies)
    def state_history(self):
        return self._view("or_state_ptr", (self.nt + 1,) + self.shape)

    def grad_state_history(self):
        return self._view("or_gradstate_ptr", (self.nt + 1, 3) + self.shape)

    def dispm(self):
        return self._view("or_dispm_ptr", (3,) + self.shape)

    def dispp(self):
        return self._view("or_dispp_ptr", (3,) + self.shape)

    def divv(self):
        return self._view("or_div_ptr", self.shape)

    def divv_at_xp(self):
        return self._view("or_divp_ptr", self.shape)

    def objective(self, v, want_m_final: bool = False):
        """Returns (J, mismatch term, regularization term[, m(1)])."""
        v = _f64(v)
        mis, reg = ctypes.c_double(0), ctypes.c_double(0)
        mf = np.empty(self.shape) if want_m_final else None
        J = lib().or_objective(self._h, _p(v), ctypes.byref(mis), ctypes.byref(reg),
                               _p(mf) if mf is not None else None)
        if want_m_final:
            return J, mis.value, reg.value, mf
        return J, mis.value, reg.value

    def gradient(self, v, want_adjoint: bool = False):
        """Reduced gradient g (Eq. 3.1) and J; linearizes at v."""
        v = _f64(v)
        g = np.empty((3,) + self.shape)
        J = ctypes.c_double(0)
        lh = np.empty((self.nt + 1,) + self.shape) if want_adjoint else None
        lib().or_gradient(self._h, _p(v), _p(g), ctypes.byref(J),
                          _p(lh) if lh is not None else None)
        if want_adjoint:
            return g, J.value, lh
        return g, J.value

    def matvec(self, vt, want_inc: bool = False):
        """GN Hessian matvec (Eq. 3.4) at the current linearization."""
        vt = _f64(vt)
        out = np.empty((3,) + self.shape)
        mt = np.empty(self.shape) if want_inc else None
        lt = np.empty((self.nt + 1,) + self.shape) if want_inc else None
        rc = lib().or_matvec(self._h, _p(vt), _p(out), _p(mt) if mt is not None else None,
                             _p(lt) if lt is not None else None)
        if rc != 0:
            raise RuntimeError("oracle matvec called before linearize/gradient")
        if want_inc:
            return out, mt, lt
        return out

    def precond(self, r):
        r = _f64(r)
        out = np.empty_like(r)
        lib().or_precond(self._h, _p(r), _p(out))
        return out

    def solve(self, v0, max_gn=50, max_pcg=100, fixed_pcg=0, eps_n=5e-2, armijo_c1=1e-4,
              max_ls=12, pc="invA", eps_h0=1e-3, max_inner=500):
        """pc: "invA", "invH0" or "2LinvH0" (Section 3 "Preconditioning")."""
        v = _f64(v0).copy()
        pcn = {"invA": 0, "invH0": 1, "2LinvH0": 2}[pc]
        o = _SolveOpts(max_gn, max_pcg, fixed_pcg, eps_n, armijo_c1, max_ls, pcn, eps_h0, max_inner)
        r = _SolveReport()
        lib().or_solve(self._h, _p(v), ctypes.byref(o), ctypes.byref(r))
        rep = SolveReport(**{k: getattr(r, k) for k, _ in _SolveReport._fields_})
        return v, rep

    def solve_continuation(self, v0, beta_target, beta_start=1.0, factor=0.1, pc="invH0",
                           **kw):
        """beta-continuation: GN solves for beta_k = max(target, start * factor^k),
        warm-started; InvA while beta_k > 0.5, pc below.  Returns (v, report,
        levels); the problem's beta is left at the target."""
        v = _f64(v0).copy()
        opts = dict(max_gn=50, max_pcg=100, fixed_pcg=0, eps_n=5e-2, armijo_c1=1e-4, max_ls=12,
                    eps_h0=1e-3, max_inner=500)
        opts.update(kw)
        pcn = {"invA": 0, "invH0": 1, "2LinvH0": 2}[pc]
        o = _SolveOpts(opts["max_gn"], opts["max_pcg"], opts["fixed_pcg"], opts["eps_n"],
                       opts["armijo_c1"], opts["max_ls"], pcn, opts["eps_h0"], opts["max_inner"])
        r = _SolveReport()
        lev = _I(0)
        lib().or_solve_continuation(self._h, _p(v), beta_target, beta_start, factor,
                                    ctypes.byref(o), ctypes.byref(r), ctypes.byref(lev))
        self.beta = beta_target
        rep = SolveReport(**{k: getattr(r, k) for k, _ in _SolveReport._fields_})
        return v, rep, int(lev.value)
