"""Pins of the oracle's alternative discretization, the paper's GPU choice:
eighth-order central differences for first derivatives (Section 4.2) and
trilinear interpolation (Section 4.1)."""
import numpy as np
import pytest

import oracle as O
from paper_2008_12820_gb300 import synth

C = np.array([4 / 5, -1 / 5, 4 / 105, -1 / 280])


def test_fd8_modified_wavenumber_closed_form():
    """FD8 maps sin(k x) to kappa(k) cos(k x) with the modified wavenumber
    kappa = (2/h) sum_j c_j sin(j k h), exactly."""
    shape = (32, 24, 40)
    x = np.meshgrid(*synth.grid_axes(shape), indexing="ij")
    for d, k in ((0, 3), (1, 7), (2, 11)):
        h = 2 * np.pi / shape[d]
        f = np.sin(k * x[d] + 0.3)
        kappa = 2 / h * sum(C[j] * np.sin((j + 1) * k * h) for j in range(4))
        g = O.grad_fd8(f)
        assert np.abs(g[d] - kappa * np.cos(k * x[d] + 0.3)).max() < 1e-12 * kappa
        for e in range(3):
            if e != d:
                assert np.abs(g[e]).max() < 1e-12


def test_fd8_is_eighth_order():
    errs = []
    for n in (16, 32):
        x = np.meshgrid(*synth.grid_axes((n, n, n)), indexing="ij")
        f = np.sin(x[0]) * np.cos(2 * x[1]) + np.sin(x[2])
        g = O.grad_fd8(f)
        ref = np.cos(x[0]) * np.cos(2 * x[1])
        errs.append(np.abs(g[0] - ref).max())
    assert errs[0] / errs[1] > 200  # 2^8 = 256


def test_fd8_divergence_is_sum_of_partials():
    shape = (16, 16, 16)
    rng = np.random.Generator(np.random.PCG64(3))
    v = synth.bandlimited_field(shape, 4, rng)
    dv = O.div_fd8(v)
    ref = sum(O.grad_fd8(v[d])[d] for d in range(3))
    assert np.abs(dv - ref).max() < 1e-12


def test_trilinear_exact_on_multilinear_and_second_order():
    n = (10, 12, 14)
    rng = np.random.default_rng(0)
    a = rng.standard_normal(8)
    I = np.meshgrid(*[np.arange(k, dtype=float) for k in n], indexing="ij")

    def p(x, y, z):
        return (a[0] + a[1] * x + a[2] * y + a[3] * z + a[4] * x * y + a[5] * y * z + a[6] * x * z
                + a[7] * x * y * z)

    f = p(*I)
    q = np.stack([rng.uniform(0, k - 1.001, 300) for k in n])
    assert np.abs(O.lerp(f, q) - p(q[0], q[1], q[2])).max() < 1e-10
    errs = []
    for N in (16, 32):
        x = np.meshgrid(*synth.grid_axes((N, N, N)), indexing="ij")
        g = np.sin(x[0]) * np.cos(x[1] - 0.2) * np.sin(x[2] + 1)
        u = rng.uniform(0, 1, (3, 200)) * N
        xq = u * 2 * np.pi / N
        ref = np.sin(xq[0]) * np.cos(xq[1] - 0.2) * np.sin(xq[2] + 1)
        errs.append(np.abs(O.lerp(g, u) - ref).max())
    assert 3 < errs[0] / errs[1] < 6  # second order: 4


def test_problem_with_fd8_and_linear_solves():
    n = 16
    w = synth.workload("sin32", shape=(n, n, n))
    P = O.Problem(w["m0"], w["m1"], 4, 1e-2, 1.0)
    P.set_discretization(interp="linear", deriv="fd8")
    g, J = P.gradient(np.zeros((3, n, n, n)))
    # at v = 0: g = (m1 - m0) FD8 grad m0 exactly
    ref = (w["m1"].astype(float) - w["m0"].astype(float))[None] * O.grad_fd8(w["m0"])
    assert np.abs(g - ref).max() < 1e-12 * np.abs(ref).max()
    v, rep = P.solve(np.zeros((3, n, n, n)))
    assert rep.status == 0 and rep.grel <= 5e-2
