"""The FP16-storage form (stored m^j, grad m^j and lambda^j in FP16, FP32
arithmetic) against the FP64 oracle and against the FP32 form on the GPU.

Tolerances follow from the FP16 unit roundoff u = 2^-11 (round to nearest
even on store).  Each stored value carries a relative error of at most u and
these errors are independent between time steps, so after j steps a field
transported by interpolation (weights summing to one) is off by about
u*sqrt(j+1) in relative L2; the tests allow 4x that.  Two quantities magnify
the stored-state rounding and get their own bound:
  * grad m^j: the rounding noise of m^j is white, and spectral differentiation
    scales white noise by the rms wavenumber (about n/2 on n points), against
    the |k| ~ 4 of the signal: rel error ~ u*sqrt(j+1)*n/8, allowed 4x;
  * lambda^j: lambda^nt = m1 - m^nt is a small difference of O(1) fields, so
    the absolute rounding of m^nt is relative to ||m(1)|| / ||lambda^nt||.
The gradient, the objective and the Hessian matvec integrate these fields and
come out far more accurate than the worst of them (measured 2e-4, 6e-6 and
1.5e-4 at 32^3); they are held to the transport bound.  A full solve in FP16
storage must take the same Gauss-Newton path as the FP32 form and land on the
same objective within the same bound."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2008_12820_gb300 import synth

pytestmark = pytest.mark.gpu

U16 = 2.0 ** -11


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def claire():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2008_12820_gb300 import claire as C
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return C


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("shape,nt", [((32, 32, 32), 4), ((48, 40, 36), 3), ((64, 64, 64), 8)])
def test_fp16_storage_operators_vs_oracle(claire, shape, nt):
    """state, grad m, adjoint, gradient, objective and matvec of one
    linearization (rows a3, a4, a6, a7-a9) in the FP16-storage form"""
    d = synth.sinusoid_pair(shape, 1000)
    m0, m1, v = d["m0"], d["m1"], (0.8 * d["v_true"]).astype(np.float32)
    vt = synth.smooth_direction(shape, 7).astype(np.float32)
    P = O.Problem(m0, m1, nt, 1e-2, 1.0)
    P.linearize(v)
    mh, gmh = P.state_history(), P.grad_state_history()
    go, Jo, lh = P.gradient(v, want_adjoint=True)
    Ho = P.matvec(vt)
    tol = 4 * U16 * math.sqrt(nt + 1)
    tol_gm = tol * max(shape) / 8
    tol_adj = tol * np.linalg.norm(mh[nt]) / np.linalg.norm(lh[nt])
    with claire.Registration(shape, nt, 1e-2, 1.0, precision="fp16") as reg:
        reg.set_images(dev(m0), dev(m1))
        g, J = reg.gradient(dev(v))
        for j in range(nt + 1):
            assert rel(host(reg.field("state", j)), mh[j]) < tol, j
            assert rel(host(reg.field("gradm", j)), gmh[j]) < tol_gm, j
            assert rel(host(reg.field("adj", j)), lh[j]) < tol_adj, j
        assert rel(host(g), go) < tol
        assert abs(J - Jo) / abs(Jo) < tol
        H = reg.hess_matvec(dev(v), dev(vt))
        assert rel(host(H), Ho) < tol


def test_fp16_storage_fixed_work_step_vs_oracle(claire):
    """sinusoid workload, 32^3: 1 GN iteration with exactly 10 PCG steps in
    the FP16-storage form against the oracle's FP64 solve"""
    w = synth.workload("sin32")
    shape, nt, beta, gamma = w["shape"], w["nt"], w["beta"], w["gamma"]
    P = O.Problem(w["m0"], w["m1"], nt, beta, gamma)
    vo, ro = P.solve(np.zeros((3,) + shape), max_gn=1, fixed_pcg=10)
    tol = 4 * U16 * math.sqrt(nt + 1)
    with claire.Registration(shape, nt, beta, gamma, precision="fp16") as reg:
        reg.set_images(dev(w["m0"]), dev(w["m1"]))
        v = torch.zeros((3,) + shape, device="cuda")
        rep = reg.solve(v, max_gn=1, fixed_pcg=10)
        assert rep.n_gn == 1 and rep.n_pcg == 10
        assert rel(host(v), vo) < tol
        assert abs(rep.J - ro.J) / abs(ro.J) < tol
        assert abs(rep.g - ro.g) / abs(ro.g) < tol


@pytest.mark.parametrize("precond", ["invA", "2LinvH0"])
def test_fp16_storage_solve_matches_fp32_form(claire, precond):
    """blob workload at 96^3 (cfg1 generator): the FP16-storage form takes the
    FP32 form's Gauss-Newton path to the same accuracy"""
    w = synth.workload("blob256", shape=(96, 96, 96))
    shape, nt, beta, gamma = w["shape"], w["nt"], w["beta"], w["gamma"]
    tol = 4 * U16 * math.sqrt(nt + 1)
    out = {}
    for prec in ("fp32", "fp16"):
        with claire.Registration(shape, nt, beta, gamma, precision=prec) as reg:
            reg.set_images(dev(w["m0"]), dev(w["m1"]))
            v = torch.zeros((3,) + shape, device="cuda")
            rep = reg.solve(v, precond=precond)
            assert rep.status == 0 and rep.grel <= 5e-2
            out[prec] = (rep, host(v))
    r32, v32 = out["fp32"]
    r16, v16 = out["fp16"]
    assert r16.n_gn == r32.n_gn and abs(r16.n_pcg - r32.n_pcg) <= 1
    assert abs(r16.J - r32.J) / abs(r32.J) < tol
    assert abs(r16.mismatch_rel - r32.mismatch_rel) / r32.mismatch_rel < tol
    assert rel(v16, v32) < tol


def test_fp16_storage_paper_gpu_discretization(claire):
    """FD8 derivatives and trilinear interpolation with FP16 storage against
    the oracle in the same discretization"""
    shape, nt = (32, 32, 32), 4
    d = synth.sinusoid_pair(shape, 1000)
    m0, m1, v = d["m0"], d["m1"], (0.8 * d["v_true"]).astype(np.float32)
    vt = synth.smooth_direction(shape, 7).astype(np.float32)
    P = O.Problem(m0, m1, nt, 1e-2, 1.0)
    P.set_discretization(interp="linear", deriv="fd8")
    go, Jo = P.gradient(v)
    Ho = P.matvec(vt)
    tol = 4 * U16 * math.sqrt(nt + 1)
    with claire.Registration(shape, nt, 1e-2, 1.0, precision="fp16") as reg:
        reg.set_discretization(interp="linear", deriv="fd8")
        reg.set_images(dev(m0), dev(m1))
        g, J = reg.gradient(dev(v))
        assert rel(host(g), go) < tol
        assert abs(J - Jo) / abs(Jo) < tol
        assert rel(host(reg.hess_matvec(dev(v), dev(vt))), Ho) < tol


def test_fp16_storage_odd_sizes_and_wide_displacement(claire):
    """n3 not a multiple of 8 (element-wise FP16 box copy) and displacements
    wider than the shared-memory box (global gather of FP16 fields)"""
    for shape, scale in [((20, 27, 45), 0.8), ((32, 32, 32), 6.0)]:
        nt = 2
        d = synth.sinusoid_pair(shape, 1001)
        m0, m1, v = d["m0"], d["m1"], (scale * d["v_true"]).astype(np.float32)
        P = O.Problem(m0, m1, nt, 1e-2, 1.0)
        P.linearize(v)
        mh = P.state_history()
        go, Jo = P.gradient(v)
        tol = 4 * U16 * math.sqrt(nt + 1)
        with claire.Registration(shape, nt, 1e-2, 1.0, precision="fp16") as reg:
            reg.set_images(dev(m0), dev(m1))
            g, J = reg.gradient(dev(v))
            for j in range(nt + 1):
                assert rel(host(reg.field("state", j)), mh[j]) < tol, (shape, j)
            assert rel(host(g), go) < tol, shape
            assert abs(J - Jo) / abs(Jo) < tol, shape


def test_fp16_storage_invalid_precision(claire):
    with pytest.raises(claire.ClaireError) as e:
        claire.Registration((8, 8, 8), 2, 1e-2, 1.0, precision=7)
    assert e.value.code == 1
