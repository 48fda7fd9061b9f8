"""Pins of the oracle's Gauss-Newton-Krylov loop (Algorithm 1, Eq. 3.3) that
do not go through its own arithmetic:

* the Armijo test: its acceptance threshold on the sufficient-decrease
  constant c1 sits where central differences of the objective (the forward
  solve alone, no gradient code) put it, and a rejected unit step is halved;
* the inexact-Newton forcing term eps_K = min(sqrt(||g_k|| / ||g_0||), 0.5):
  each Gauss-Newton step takes exactly as many PCG iterations as SciPy's
  conjugate-gradient routine needs, with the same operator and the inverse-A
  preconditioner, to reach that relative residual; the linear and constant
  alternatives give other counts on this problem.

CPU only (FP64 oracle, 32^3 sinusoid problem)."""
import numpy as np
import pytest

import oracle as O
from paper_2008_12820_gb300 import synth

sla = pytest.importorskip("scipy.sparse.linalg")

SHAPE, NT, BETA, GAMMA = (32, 32, 32), 4, 1e-2, 1.0


def problem():
    d = synth.sinusoid_pair(SHAPE, 1000)
    return d["m0"].astype(float), d["m1"].astype(float)


def test_armijo_threshold_and_halving():
    """One GN step with one PCG iteration from v = 0: the direction is the
    line minimiser of the GN model along z = (beta A)^-1 (-g).  With
    rho = (J(v + vt) - J(v)) / J'(v; vt), J' by central differences, the step
    is accepted at alpha = 1 for c1 just below rho and halved (then accepted,
    J at alpha = 1/2 decreasing by more) for c1 just above.  A sign error in
    the slope, a missing h^3 weight or another backtracking factor moves the
    threshold or the step."""
    m0, m1 = problem()
    P = O.Problem(m0, m1, NT, BETA, GAMMA)
    v0 = np.zeros((3,) + SHAPE)
    g, J0 = P.gradient(v0)
    z = O.apply_Ainv(-g, BETA, GAMMA)
    alpha = np.sum(-g * z) / np.sum(z * P.matvec(z))   # first PCG iterate, x0 = 0
    vt = alpha * z
    eps = 1e-4
    slope = (P.objective(v0 + eps * vt)[0] - P.objective(v0 - eps * vt)[0]) / (2 * eps)
    assert slope < 0
    rho = (P.objective(v0 + vt)[0] - J0) / slope
    rho_half = (P.objective(v0 + 0.5 * vt)[0] - J0) / (0.5 * slope)
    # a descent step of the GN model: rho near 1/2, and larger for the half step
    assert 0.2 < rho < 0.9 and rho_half > rho * 1.1
    # the gradient's slope differs from the central difference by the OTD
    # discretization gap (< 1% here); 2% margins stay clear of it
    v, rep = P.solve(v0, max_gn=1, fixed_pcg=1, armijo_c1=0.98 * rho)
    assert rep.n_gn == 1 and rep.status == 0
    assert np.linalg.norm(v - vt) < 1e-10 * np.linalg.norm(vt)
    v, rep = P.solve(v0, max_gn=1, fixed_pcg=1, armijo_c1=1.02 * rho)
    assert rep.n_gn == 1 and rep.status == 0
    assert np.linalg.norm(v - 0.5 * vt) < 1e-10 * np.linalg.norm(vt)


def cg_count(P, g, rtol):
    """iterations SciPy's preconditioned CG needs from x0 = 0 to reach
    ||r|| <= rtol ||r0|| on H x = -g, and its solution"""
    n = g.size
    H = sla.LinearOperator((n, n), matvec=lambda x: P.matvec(x.reshape(g.shape)).ravel())
    M = sla.LinearOperator((n, n), matvec=lambda x: O.apply_Ainv(x.reshape(g.shape), BETA, GAMMA).ravel())
    it = [0]

    def cb(xk):
        it[0] += 1

    x, info = sla.cg(H, -g.ravel(), rtol=rtol, M=M, callback=cb, maxiter=100)
    assert info == 0
    return it[0], x.reshape(g.shape)


def test_forcing_term_against_scipy_cg():
    m0, m1 = problem()
    v0 = np.zeros((3,) + SHAPE)
    runs = [O.Problem(m0, m1, NT, BETA, GAMMA).solve(v0, max_gn=k) for k in (1, 2, 3)]
    P = O.Problem(m0, m1, NT, BETA, GAMMA)
    prev_pcg, prev_v, prev_grel = 0, v0, 1.0
    for k, (v, rep) in enumerate(runs, start=1):
        assert rep.n_gn == k and rep.status == 0
        steps = rep.n_pcg - prev_pcg
        g, _ = P.gradient(prev_v)   # linearizes at the iterate of step k
        tol = min(np.sqrt(prev_grel), 0.5)
        want, x = cg_count(P, g, tol)
        assert steps == want, (k, steps, want)
        if k == 1:
            # unit step accepted: the first iterate is v0 + the CG solution
            assert np.linalg.norm(v - (v0 + x)) < 1e-8 * np.linalg.norm(x)
        if k == 3:
            # on this step the alternatives take other counts
            assert cg_count(P, g, min(prev_grel, 0.5))[0] != want
            assert cg_count(P, g, 0.5)[0] != want
        prev_pcg, prev_v, prev_grel = rep.n_pcg, v, rep.grel
