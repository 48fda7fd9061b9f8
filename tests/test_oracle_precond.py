"""Pins of the oracle's zero-velocity Hessian preconditioners (Section 3,
"Preconditioning"; Algorithm 2): H0 against the Gauss-Newton Hessian at
v = 0, the inner PCG against a dense direct solve, spectral restriction and
prolongation against band-limited closed forms, and the closed form of both
variants when grad m vanishes."""
import numpy as np
import pytest

import oracle as O
from paper_2008_12820_gb300 import synth


def trig(shape, modes):
    x = np.meshgrid(*synth.grid_axes(shape), indexing="ij")
    f = np.zeros(shape)
    for (k1, k2, k3), a, ph in modes:
        f += a * np.cos(k1 * x[0] + k2 * x[1] + k3 * x[2] + ph)
    return f


def test_h0_is_the_gauss_newton_hessian_at_zero_velocity():
    shape = (12, 10, 14)
    d = synth.sinusoid_pair(shape, 1000)
    m0, m1 = d["m0"].astype(float), d["m1"].astype(float)
    beta, gamma = 0.1, 1.0
    P = O.Problem(m0, m1, 4, beta, gamma)
    P.gradient(np.zeros((3,) + shape))
    vt = synth.smooth_direction(shape, 4).astype(float)
    ref = P.matvec(vt)
    got = O.h0_matvec(vt, O.grad(m0), beta, gamma)
    assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max()


def test_invh0_matches_dense_solve_8cubed():
    shape = (8, 8, 8)
    rng = np.random.default_rng(0)
    m = synth.sinusoid_pair(shape, 1001)["m0"].astype(float)
    gm = O.grad(m)
    n = 3 * 512
    H = np.empty((n, n))
    e = np.zeros(n)
    for i in range(n):
        e[:] = 0
        e[i] = 1
        H[:, i] = O.h0_matvec(e.reshape((3,) + shape), gm, 5e-2, 1.0).ravel()
    assert np.abs(H - H.T).max() < 1e-12 * np.abs(H).max()
    assert np.linalg.eigvalsh(H).min() > 0
    r = rng.standard_normal((3,) + shape)
    s, it = O.invh0(r, gm, 5e-2, 1.0, 1e-12, maxit=2000)
    ref = np.linalg.solve(H, r.ravel()).reshape(r.shape)
    assert np.abs(s - ref).max() < 1e-8 * np.abs(ref).max()


def test_restriction_and_prolongation_are_exact_on_band_limited_fields():
    fine, coarse = (24, 20, 16), (12, 10, 8)
    low = [((1, -2, 3), 0.7, 0.3), ((-5, 4, 1), 1.1, 1.0), ((0, 0, 2), 0.4, -0.5)]
    high = [((6, 1, 0), 0.9, 0.2), ((1, 5, 4), 0.5, 0.0)]  # |k_d| >= nc_d/2 in some axis
    f_low_fine, f_low_coarse = trig(fine, low), trig(coarse, low)
    # prolongation interpolates band-limited coarse data exactly
    assert np.abs(O.prolong(f_low_coarse, fine) - f_low_fine).max() < 1e-12
    # restriction samples band-limited fine data exactly and drops the rest
    f = f_low_fine + trig(fine, high)
    assert np.abs(O.restrict(f, coarse) - f_low_coarse).max() < 1e-12
    assert np.abs(O.restrict(O.prolong(f_low_coarse, fine), coarse) - f_low_coarse).max() < 1e-12
    # the high-pass part is what the coarse grid cannot hold
    assert np.abs(O.highpass(f, coarse) - trig(fine, high)).max() < 1e-12


def test_both_variants_reduce_to_inverse_A_without_image_gradient():
    shape = (16, 12, 20)
    rng = np.random.default_rng(1)
    r = rng.standard_normal((3,) + shape)
    r -= r.mean(axis=(1, 2, 3), keepdims=True)  # H0 = beta A is singular on constants
    gm = np.zeros((3,) + shape)
    ref = O.apply_Ainv(r, 5e-2, 1.0)
    s1, it1 = O.invh0(r, gm, 5e-2, 1.0, 1e-12)
    assert it1 == 1 and np.abs(s1 - ref).max() < 1e-10 * np.abs(ref).max()
    s2, _ = O.invh0(r, gm, 5e-2, 1.0, 1e-12, two_level=True)
    assert np.abs(s2 - ref).max() < 1e-10 * np.abs(ref).max()


def test_zero_velocity_preconditioners_cut_outer_pcg_iterations():
    """Section 5.1: fewer PCG iterations than the spectral preconditioner."""
    n = 32
    w = synth.workload("blob256", shape=(n, n, n))
    P = O.Problem(w["m0"], w["m1"], 4, 1e-2, 1.0)
    _, ra = P.solve(np.zeros((3, n, n, n)), pc="invA")
    _, rh = P.solve(np.zeros((3, n, n, n)), pc="invH0")
    _, r2 = P.solve(np.zeros((3, n, n, n)), pc="2LinvH0")
    for r in (ra, rh, r2):
        assert r.status == 0 and r.grel <= 5e-2
    assert rh.n_pcg < ra.n_pcg and r2.n_pcg < ra.n_pcg
    assert rh.n_inner > 0 and r2.n_inner > 0


def test_beta_continuation():
    """Section 3: a decreasing sequence of beta, each level warm-started; with
    the start at the target it is exactly one solve."""
    n = 16
    w = synth.workload("sin32", shape=(n, n, n))
    P = O.Problem(w["m0"], w["m1"], 4, 1e-2, 1.0)
    v1, r1 = P.solve(np.zeros((3, n, n, n)), pc="invH0")
    v2, r2, lev = P.solve_continuation(np.zeros((3, n, n, n)), 1e-2, beta_start=1e-2, pc="invH0")
    assert lev == 1 and np.array_equal(v1, v2) and r1.J == r2.J
    v3, r3, lev = P.solve_continuation(np.zeros((3, n, n, n)), 1e-2, beta_start=1.0, factor=0.1,
                                       pc="invH0")
    assert lev == 3 and r3.status == 0 and r3.grel <= 5e-2
    # the target-level objective at the continuation's result matches a direct
    # solve to the GN tolerance (both are stationary points of the same J)
    P.beta = 1e-2
    J3, _, _ = P.objective(v3)
    assert abs(J3 - r1.J) / r1.J < 0.05
