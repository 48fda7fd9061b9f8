"""Pins of the oracle's periodic cubic Lagrange interpolation (paper
Section 4.1: f(x) = sum_{ijk} f_ijk phi_i(x1) phi_j(x2) phi_k(x3) with Lagrange
basis polynomials, degree 3 here)."""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2008_12820_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lagrange_cubic_weights.txt")


def read_golden():
    rows = []
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if line:
            rows.append([float(Fraction(t)) for t in line.split()])
    return rows


def test_lagrange_weights_match_hand_worked_values():
    for t, *w in read_golden():
        got = [O.lagrange(a, t) for a in (-1, 0, 1, 2)]
        assert np.allclose(got, w, rtol=0, atol=1e-15), (t, got, w)


def test_lagrange_weights_reproduce_monomials():
    # sum_a a^p phi_a(t) = t^p for p <= 3 (exactness of cubic Lagrange)
    for t in np.linspace(0, 1, 11):
        for p in range(4):
            s = sum((a ** p) * O.lagrange(a, t) for a in (-1, 0, 1, 2))
            assert abs(s - t ** p) < 1e-14


def test_reproduces_tensor_cubic_polynomials_without_wrap():
    n = (16, 14, 12)
    rng = np.random.default_rng(0)
    C = rng.standard_normal((4, 4, 4))
    I1, I2, I3 = np.meshgrid(*[np.arange(k, dtype=float) for k in n], indexing="ij")

    def p(a, b, c):
        return sum(C[i, j, k] * a ** i * b ** j * c ** k
                   for i in range(4) for j in range(4) for k in range(4))

    f = p(I1, I2, I3)
    # queries whose stencil floor(q)-1 .. floor(q)+2 stays inside the grid
    q = np.stack([rng.uniform(1, nn - 3, 500) for nn in n])
    got = O.interp(f, q)
    ref = p(q[0], q[1], q[2])
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


def test_exact_at_grid_nodes_and_periodic():
    n = (8, 9, 10)
    rng = np.random.default_rng(1)
    f = rng.standard_normal(n)
    I = np.stack(np.meshgrid(*[np.arange(k, dtype=float) for k in n], indexing="ij")).reshape(3, -1)
    assert np.abs(O.interp(f, I) - f.ravel()).max() < 1e-14
    # a shift by a whole period in any axis gives the same value
    q = np.stack([rng.uniform(-2, k + 2, 200) for k in n])
    base = O.interp(f, q)
    for d in range(3):
        qs = q.copy()
        qs[d] += n[d]
        assert np.abs(O.interp(f, qs) - base).max() < 1e-12
        qs[d] -= 3 * n[d]
        assert np.abs(O.interp(f, qs) - base).max() < 1e-12


def test_fourth_order_convergence_on_smooth_periodic_function():
    errs = []
    rng = np.random.default_rng(2)
    u = rng.uniform(0, 1, (3, 400))
    for N in (16, 32, 64):
        x = synth.grid_axes((N, N, N))
        X = np.meshgrid(*x, indexing="ij")
        f = np.sin(X[0]) * np.cos(2 * X[1]) * np.sin(X[2] + 1)
        q = u * N  # index units
        xq = q * (2 * np.pi / N)
        ref = np.sin(xq[0]) * np.cos(2 * xq[1]) * np.sin(xq[2] + 1)
        errs.append(np.abs(O.interp(f, q) - ref).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 12 < r1 < 20 and 12 < r2 < 20, errs
