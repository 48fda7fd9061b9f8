"""Pins of the oracle's FFT and spectral operators (paper Section 3,
"Discretization": spectral vector Laplacian, divergence penalty and the
inverse used by the preconditioner of Section 3, "Preconditioning").

Each check compares the oracle with something other than itself: a
brute-force DFT, numpy's FFT, derivatives of trigonometric polynomials in
closed form, the closed-form symbol on single Fourier modes, and integration
by parts identities."""
import numpy as np
import pytest

import oracle as O
from paper_2008_12820_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore")


def brute_dft3(a, sign):
    out = np.asarray(a, dtype=np.complex128)
    for axis, n in enumerate(a.shape):
        j = np.arange(n)
        F = np.exp(sign * 2j * np.pi * np.outer(j, j) / n)
        out = np.moveaxis(np.tensordot(F, np.moveaxis(out, axis, 0), axes=(1, 0)), 0, axis)
    return out


@pytest.mark.parametrize("shape", [(8, 8, 8), (6, 6, 6), (10, 10, 10), (15, 15, 15), (4, 6, 10),
                                   (9, 5, 12)])
def test_fft_matches_bruteforce_dft(shape):
    rng = np.random.default_rng(1)
    a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    for sign in (-1, +1):
        ref = brute_dft3(a, sign)
        got = O.fft3(a, sign)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_fft_matches_numpy():
    rng = np.random.default_rng(2)
    a = rng.standard_normal((30, 24, 20))
    assert np.allclose(O.fft3(a, -1), np.fft.fftn(a), rtol=0, atol=1e-10)
    assert np.allclose(O.fft3(a, +1) / a.size, np.fft.ifftn(a), rtol=0, atol=1e-13)


def trig_poly(shape, rng, nterms=6):
    """f = sum a sin(k.x + phi) with |k_d| < N_d/2, and its exact gradient."""
    x = np.meshgrid(*synth.grid_axes(shape), indexing="ij")
    f = np.zeros(shape)
    g = np.zeros((3,) + shape)
    for _ in range(nterms):
        k = [rng.integers(-(n // 2) + 1, n // 2) for n in shape]
        a, phi = rng.uniform(0.5, 1.5), rng.uniform(0, 2 * np.pi)
        ph = k[0] * x[0] + k[1] * x[1] + k[2] * x[2] + phi
        f += a * np.sin(ph)
        for d in range(3):
            g[d] += a * k[d] * np.cos(ph)
    return f, g


@pytest.mark.parametrize("shape", [(16, 16, 16), (12, 10, 18), (15, 9, 10)])
def test_gradient_exact_on_trig_polynomials(shape):
    rng = np.random.default_rng(3)
    f, g = trig_poly(shape, rng)
    assert np.abs(O.grad(f) - g).max() <= 1e-11 * np.abs(g).max()


def test_divergence_exact_on_trig_fields():
    shape = (12, 14, 16)
    rng = np.random.default_rng(4)
    v = np.zeros((3,) + shape)
    dv = np.zeros(shape)
    for d in range(3):
        f, g = trig_poly(shape, rng, 4)
        v[d] = f
        dv += g[d]
    assert np.abs(O.div(v) - dv).max() <= 1e-11 * np.abs(dv).max()


def test_nyquist_mode_has_zero_first_derivative():
    # reading: the Nyquist cosine of an even axis has no resolvable derivative
    shape = (8, 8, 8)
    x1 = synth.grid_axes(shape)[0]
    f = np.cos(4 * x1)[:, None, None] * np.ones(shape)
    assert np.abs(O.grad(f)).max() < 1e-12


@pytest.mark.parametrize("k,j", [((1, 2, -3), 0), ((2, 0, 1), 1), ((-1, 3, 2), 2), ((0, 0, 5), 2)])
def test_A_on_single_fourier_mode(k, j):
    """v = e_j cos(k.x):  beta*A v = beta|k|^2 e_j cos(k.x) + gamma k_j k cos(k.x)
    (vector Laplacian plus -gamma grad div)."""
    shape = (12, 12, 12)
    beta, gamma = 0.3, 1.7
    x = np.meshgrid(*synth.grid_axes(shape), indexing="ij")
    c = np.cos(k[0] * x[0] + k[1] * x[1] + k[2] * x[2])
    v = np.zeros((3,) + shape)
    v[j] = c
    expect = np.zeros_like(v)
    k2 = sum(kk * kk for kk in k)
    expect[j] += beta * k2 * c
    for d in range(3):
        expect[d] += gamma * k[j] * k[d] * c
    assert np.abs(O.apply_A(v, beta, gamma) - expect).max() < 1e-10 * max(1, np.abs(expect).max())


def test_A_energy_is_h1_seminorm_plus_divergence_penalty():
    """<v, beta*A v> = beta sum_d ||grad v_d||^2 + gamma ||div v||^2 (integration
    by parts) for a band-limited v; gradients/divergence from the oracle's own
    first-derivative operators, a different code path than the symbol."""
    shape = (16, 16, 16)
    rng = np.random.Generator(np.random.PCG64(5))
    v = synth.bandlimited_field(shape, 4, rng)
    beta, gamma = 0.05, 2.0
    lhs = np.sum(v * O.apply_A(v, beta, gamma))
    rhs = beta * sum(np.sum(O.grad(v[d]) ** 2) for d in range(3)) + gamma * np.sum(O.div(v) ** 2)
    assert abs(lhs - rhs) <= 1e-11 * abs(rhs)


def test_Ainv_inverts_A_up_to_the_mean():
    shape = (10, 12, 8)
    rng = np.random.default_rng(6)
    v = rng.standard_normal((3,) + shape)
    beta, gamma = 1e-2, 1.0
    mean = v.mean(axis=(1, 2, 3), keepdims=True)
    w = O.apply_Ainv(O.apply_A(v, beta, gamma), beta, gamma)
    # A annihilates constants; the inverse is the identity on k = 0
    assert np.abs(w - (v - mean)).max() < 1e-9
    w2 = O.apply_A(O.apply_Ainv(v, beta, gamma), beta, gamma)
    assert np.abs(w2 - (v - mean)).max() < 1e-9


def test_A_and_Ainv_symmetric():
    shape = (8, 10, 12)
    rng = np.random.default_rng(7)
    u = rng.standard_normal((3,) + shape)
    w = rng.standard_normal((3,) + shape)
    for op in (O.apply_A, O.apply_Ainv):
        a = np.sum(op(u, 0.1, 0.7) * w)
        b = np.sum(u * op(w, 0.1, 0.7))
        assert abs(a - b) <= 1e-11 * (abs(a) + abs(b))


def test_Ainv_large_gamma_gives_divergence_free_field():
    """As gamma grows, (beta A)^{-1} r tends to the Leray projection of
    (-beta Laplace)^{-1} r: divergence-free."""
    shape = (12, 12, 12)
    rng = np.random.Generator(np.random.PCG64(8))
    r = synth.bandlimited_field(shape, 4, rng)
    s = O.apply_Ainv(r, 1.0, 1e9)
    s0 = O.apply_Ainv(r, 1.0, 0.0)
    assert np.abs(O.div(s)).max() < 1e-7 * np.abs(O.div(s0)).max()
