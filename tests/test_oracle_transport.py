"""Pins of the oracle's transport solves, reduced gradient (Eq. 3.1), adjoint
(Eq. 3.2), Gauss-Newton Hessian matvec (Eqs. 3.4-3.6), PCG and the
Gauss-Newton-Krylov solver (Algorithm 1, Eq. 3.3).

The gradient and Hessian are optimize-then-discretize: they are not exact
derivatives of the discrete objective, so FD and symmetry checks hold up to a
discretization gap that must shrink under refinement.  Two special cases are
exact: v = 0 (closed forms, the H0 of Section 3 "Preconditioning") and a
constant velocity that moves every characteristic by whole grid cells per
time step (transport is then a permutation and the adjoint its transpose)."""
import numpy as np
import pytest

import oracle as O
from paper_2008_12820_gb300 import synth

TWO_PI = 2 * np.pi


def smooth_pair(shape, seed=1000):
    d = synth.sinusoid_pair(shape, seed)
    return d["m0"].astype(float), d["m1"].astype(float), d["v_true"].astype(float)


def h3(shape):
    return np.prod([TWO_PI / n for n in shape])


# ------------------------------------------------------------------ v = 0 ---

def test_zero_velocity_closed_forms():
    shape, nt, beta, gamma = (12, 10, 14), 4, 1e-2, 1.0
    m0, m1, _ = smooth_pair(shape)
    P = O.Problem(m0, m1, nt, beta, gamma)
    v = np.zeros((3,) + shape)
    g, J = P.gradient(v)
    assert np.abs(P.dispm()).max() == 0 and np.abs(P.dispp()).max() == 0
    assert np.abs(P.state_history() - m0[None]).max() < 1e-14
    gm0 = O.grad(m0)
    # g = (m1 - m0) grad m0 exactly
    assert np.abs(g - (m1 - m0)[None] * gm0).max() < 1e-12
    assert abs(J - 0.5 * h3(shape) * np.sum((m1 - m0) ** 2)) < 1e-12
    # H(0) vt = beta A vt + grad m0 (grad m0 . vt) = H0 vt
    vt = synth.smooth_direction(shape, 3).astype(float)
    Hv = P.matvec(vt)
    H0v = O.apply_A(vt, beta, gamma) + gm0 * np.sum(gm0 * vt, axis=0)[None]
    assert np.abs(Hv - H0v).max() < 1e-11 * np.abs(H0v).max()


# ------------------------------------------------ integer-shift velocity ---

def shift_problem(shape=(12, 12, 12), nt=4, s=(1, -2, 1), beta=1e-2, gamma=1.0):
    m0, m1, _ = smooth_pair(shape, 1003)
    c = [s[d] * (TWO_PI / shape[d]) * nt for d in range(3)]  # dt * c_d = s_d * h_d
    v = np.stack([np.full(shape, c[d]) for d in range(3)])
    P = O.Problem(m0, m1, nt, beta, gamma)
    return P, v, m0, m1, s


def test_integer_shift_is_exact_permutation():
    P, v, m0, m1, s = shift_problem()
    P.gradient(v)
    for d in range(3):
        assert np.abs(P.dispm()[d] + s[d]).max() < 1e-12
        assert np.abs(P.dispp()[d] - s[d]).max() < 1e-12
    mh = P.state_history()
    for j in range(P.nt + 1):
        ref = np.roll(m0, shift=tuple(j * si for si in s), axis=(0, 1, 2))
        assert np.abs(mh[j] - ref).max() < 1e-12


def test_integer_shift_adjoint_identities_exact():
    P, v, m0, m1, s = shift_problem()
    g, _ = P.gradient(v)
    b = g - O.apply_A(v, P.beta, P.gamma)
    vt = synth.smooth_direction(P.shape, 11).astype(float)
    _, _, _, mf = P.objective(v, want_m_final=True)
    Hv, mt, _ = P.matvec(vt, want_inc=True)
    bt = Hv - O.apply_A(vt, P.beta, P.gamma)
    # <int lambda grad m, vt> = <m(1) - m1, mt(1)>  and  <int lt grad m, vt> = ||mt(1)||^2
    a1, a2 = np.sum(b * vt), np.sum((mf - m1) * mt)
    assert abs(a1 - a2) < 1e-11 * abs(a2)
    c1, c2 = np.sum(bt * vt), np.sum(mt * mt)
    assert abs(c1 - c2) < 1e-11 * abs(c2)


def test_integer_shift_hessian_dense_symmetric_psd_and_pcg_matches_direct_solve():
    """Brute force on an 8^3 grid: assemble the 1536 x 1536 matrix from matvecs."""
    P, v, m0, m1, s = shift_problem(shape=(8, 8, 8), nt=4, s=(1, 0, -1))
    P.gradient(v)
    n = 3 * P.N
    H = np.empty((n, n))
    e = np.zeros(n)
    for i in range(n):
        e[:] = 0
        e[i] = 1
        H[:, i] = P.matvec(e.reshape((3,) + P.shape)).ravel()
    assert np.abs(H - H.T).max() < 1e-12 * np.abs(H).max()
    ev = np.linalg.eigvalsh(0.5 * (H + H.T))
    assert ev.min() > 0  # data term makes the constant modes of A definite
    # data part is PSD: H - beta*A >= 0
    A = np.empty((n, n))
    for i in range(n):
        e[:] = 0
        e[i] = 1
        A[:, i] = O.apply_A(e.reshape((3,) + P.shape), P.beta, P.gamma).ravel()
    assert np.linalg.eigvalsh(0.5 * ((H - A) + (H - A).T)).min() > -1e-10
    # PCG (identity preconditioner) run to convergence equals the direct solve
    rng = np.random.default_rng(0)
    b = rng.standard_normal(n)
    x, it, flag, rel = O.pcg_dense(H, np.eye(n), b, 1e-12, 5 * n)
    assert flag == 0 and rel <= 1e-12
    xd = np.linalg.solve(H, b)
    assert np.abs(x - xd).max() < 1e-8 * np.abs(xd).max()


def test_constant_noninteger_velocity_converges_at_fourth_order():
    """Straight characteristics: RK2 is exact, m(1) = m0(x - c) analytically;
    the only error is interpolation, O(h^4)."""
    errs = []
    c = np.array([0.37, -0.81, 0.55])
    for N in (16, 32, 64):
        shape = (N, N, N)
        x = np.meshgrid(*synth.grid_axes(shape), indexing="ij")

        def m0f(x1, x2, x3):
            return np.sin(x1) * np.cos(x2 + 0.3) + 0.5 * np.sin(2 * x3 - x1)

        m0 = m0f(*x)
        ref = m0f(x[0] - c[0], x[1] - c[1], x[2] - c[2])
        v = np.stack([np.full(shape, c[d]) for d in range(3)])
        dm = O.footpoints(v, 4, -1)
        mh = O.state(dm, m0, 4)
        errs.append(np.abs(mh[-1] - ref).max())
    assert errs[0] / errs[1] > 10 and errs[1] / errs[2] > 12, errs


# --------------------------------------------------------- generic v -------

def test_gradient_matches_central_fd_within_discretization_gap():
    gaps = {}
    for N in (16, 32):
        shape = (N, N, N)
        m0, m1, vtrue = smooth_pair(shape)
        P = O.Problem(m0, m1, 4, 1e-2, 1.0)
        v = 0.8 * vtrue
        g, J = P.gradient(v)
        for seed in (7, 9):
            vt = synth.smooth_direction(shape, seed, kmax=3).astype(float)
            eps = 1e-4
            fd = (P.objective(v + eps * vt)[0] - P.objective(v - eps * vt)[0]) / (2 * eps)
            an = h3(shape) * np.sum(g * vt)
            gaps[N, seed] = abs(fd - an) / abs(fd)
    for seed in (7, 9):
        assert gaps[16, seed] < 2e-2 and gaps[32, seed] < 2e-3, gaps
        assert gaps[32, seed] < gaps[16, seed] / 4, gaps


def test_discretization_gaps_shrink_under_refinement():
    """Adjoint consistency <b, vt> vs <m(1)-m1, mt(1)>, mt(1) vs the central
    difference of m(1), and Hessian symmetry, at 16^3 and 32^3."""
    res = {}
    for N in (16, 32):
        shape = (N, N, N)
        m0, m1, vtrue = smooth_pair(shape)
        P = O.Problem(m0, m1, 4, 1e-2, 1.0)
        v = 0.8 * vtrue
        g, _ = P.gradient(v)
        vt = synth.smooth_direction(shape, 7, kmax=3).astype(float)
        w = synth.smooth_direction(shape, 8, kmax=3).astype(float)
        b = g - O.apply_A(v, 1e-2, 1.0)
        _, _, _, mf = P.objective(v, want_m_final=True)
        Hv, mt, _ = P.matvec(vt, want_inc=True)
        Hw = P.matvec(w)
        adj = abs(np.sum(b * vt) - np.sum((mf - m1) * mt)) / abs(np.sum(b * vt))
        eps = 1e-4
        fdm = (P.objective(v + eps * vt, True)[3] - P.objective(v - eps * vt, True)[3]) / (2 * eps)
        inc = np.linalg.norm(fdm - mt) / np.linalg.norm(fdm)
        sym = abs(np.sum(Hv * w) - np.sum(vt * Hw)) / (np.linalg.norm(Hv) * np.linalg.norm(w))
        res[N] = (adj, inc, sym)
    # third-order consistent (derivative of the cubic interpolant): x8 per halving
    assert res[32][0] < res[16][0] / 4, res
    assert res[32][1] < res[16][1] / 4, res
    assert res[16][2] < 1e-4 and res[32][2] < res[16][2], res
    assert res[32][1] < 0.05, res


def test_syn_divergence_free_velocity_gives_unit_jacobian():
    """Paper Section 5, dataset SYN: the velocity is divergence free, so the
    deformation map preserves volume: det grad y -> 1 under refinement."""
    errs = []
    for N, nt in ((16, 4), (32, 8)):
        shape = (N, N, N)
        v = synth.syn_velocity(shape).astype(float)
        assert np.abs(O.div(v)).max() < 1e-12
        det = O.det_grad_y(v, nt)
        errs.append(np.abs(det - 1).max())
    assert errs[0] < 5e-2 and errs[1] < errs[0] / 4, errs


# ---------------------------------------------------------------- PCG ------

def test_pcg_on_dense_spd_system():
    rng = np.random.default_rng(3)
    n = 60
    Q = rng.standard_normal((n, n))
    H = Q @ Q.T + n * np.eye(n)
    b = rng.standard_normal(n)
    x, it, flag, rel = O.pcg_dense(H, np.eye(n), b, 1e-12, 500)
    assert flag == 0 and np.allclose(x, np.linalg.solve(H, b), atol=1e-9)
    # the exact inverse as preconditioner converges in one iteration
    x, it, flag, rel = O.pcg_dense(H, np.linalg.inv(H), b, 1e-10, 50)
    assert it == 1 and np.allclose(x, np.linalg.solve(H, b), atol=1e-9)
    # fixed iteration count runs exactly that many
    x, it, flag, rel = O.pcg_dense(H, np.eye(n), b, 1e-30, 7, fixed=True)
    assert it == 7 and flag == 0


def test_pcg_stops_on_negative_curvature():
    n = 5
    H = np.diag([1.0, -2.0, 3.0, 4.0, 5.0])
    b = np.ones(n)
    x, it, flag, rel = O.pcg_dense(H, np.eye(n), b, 1e-12, 50)
    assert flag == 1


def test_pcg_with_exact_H0_inverse_on_zero_velocity_problem():
    """At v = 0 the GN Hessian is H0 = beta A + grad m0 (x) grad m0 (Section 3,
    'Preconditioning'); PCG preconditioned with its exact inverse converges in
    one iteration to the direct solution (8^3 brute force)."""
    shape = (8, 8, 8)
    m0, m1, _ = smooth_pair(shape)
    P = O.Problem(m0, m1, 4, 1e-1, 1.0)
    g, _ = P.gradient(np.zeros((3,) + shape))
    n = 3 * P.N
    H = np.empty((n, n))
    e = np.zeros(n)
    for i in range(n):
        e[:] = 0
        e[i] = 1
        H[:, i] = P.matvec(e.reshape((3,) + shape)).ravel()
    x, it, flag, rel = O.pcg_dense(H, np.linalg.inv(H), -g.ravel(), 1e-8, 10)
    assert it == 1
    assert np.allclose(x, np.linalg.solve(H, -g.ravel()), atol=1e-8)


# -------------------------------------------------------------- solver -----

def test_gauss_newton_decreases_objective_and_gradient():
    shape = (16, 16, 16)
    m0, m1, _ = smooth_pair(shape)
    P = O.Problem(m0, m1, 4, 1e-2, 1.0)
    v, rep = P.solve(np.zeros((3,) + shape), max_gn=5)
    assert rep.status == 0
    assert rep.J < rep.J0 and rep.grel < 1.0
    assert rep.mismatch_rel < 0.5
    # the report's J is the objective at the returned v
    J, _, _ = P.objective(v)
    assert abs(J - rep.J) < 1e-12 * abs(J)


def test_fixed_work_solve_counts():
    shape = (12, 12, 12)
    m0, m1, _ = smooth_pair(shape)
    P = O.Problem(m0, m1, 4, 1e-2, 1.0)
    v, rep = P.solve(np.zeros((3,) + shape), max_gn=1, fixed_pcg=10)
    assert rep.n_gn == 1 and rep.n_pcg == 10 and rep.n_matvec == 10


def test_rk2_footpoints_have_third_order_local_error():
    """Heun's method for dy/dt = v(y), y(t+dt) = x: local error O(dt^3).  The
    reference integrates the analytic SYN velocity backward with 200 RK4
    substeps; the grid is fine enough that interpolating v is not the limit."""
    shape = (64, 64, 64)
    h = TWO_PI / 64
    v = synth.syn_velocity(shape).astype(float)

    def vel(y):
        x1, x2, x3 = y
        return np.stack([np.sin(x3) * np.cos(x2) * np.sin(x2),
                         np.sin(x1) * np.cos(x3) * np.sin(x3),
                         np.sin(x2) * np.cos(x1) * np.sin(x1)])

    rng = np.random.default_rng(5)
    idx = rng.integers(0, 64, (3, 200))
    errs = []
    for nt in (2, 4, 8):
        dt = 1.0 / nt
        disp = O.footpoints(v, nt, -1)
        got = np.stack([disp[d][idx[0], idx[1], idx[2]] for d in range(3)]) * h
        y = idx * h
        ns = 200
        s = dt / ns
        for _ in range(ns):  # backward in time: dy/ds = -v(y)
            k1 = -vel(y)
            k2 = -vel(y + 0.5 * s * k1)
            k3 = -vel(y + 0.5 * s * k2)
            k4 = -vel(y + s * k3)
            y = y + s / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        errs.append(np.abs(got - (y - idx * h)).max())
    assert errs[0] / errs[1] > 6 and errs[1] / errs[2] > 6, errs
