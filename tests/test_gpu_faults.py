"""Failure paths of the C ABI, each made on the host side: a cap on the device
bytes a context may allocate (CLAIRE_ERR_OOM, at creation and at a later lazy
allocation), a NaN in an image (CLAIRE_ERR_NONFINITE), and a sufficient
decrease constant no step of the line search can meet within its halvings
(CLAIRE_ERR_LINESEARCH).  The velocities stay finite in every run, so every
kernel sees finite foot points; the context is used again after each error."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2008_12820_gb300 import synth

pytestmark = pytest.mark.gpu

OOM, NONFINITE, LINESEARCH = 2, 5, 6


@pytest.fixture(scope="module")
def claire():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2008_12820_gb300 import claire as C
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return C


def sin32():
    w = synth.workload("sin32")
    return w, torch.from_numpy(w["m0"]).cuda(), torch.from_numpy(w["m1"]).cuda()


def test_workspace_limit_reports_oom(claire):
    w, m0, m1 = sin32()
    shape, nt = w["shape"], w["nt"]
    with claire.Registration(shape, nt, w["beta"], w["gamma"]) as reg:
        full = reg.workspace_bytes()
    v = (0.5 * torch.from_numpy(w["v_true"])).float().cuda()
    try:
        # creation needs more than the cap
        claire.set_workspace_limit(full // 2)
        with pytest.raises(claire.ClaireError) as e:
            claire.Registration(shape, nt, w["beta"], w["gamma"])
        assert e.value.code == OOM and "workspace limit" in str(e.value)
        # creation fits; the checkpoints of the differentiable form do not
        claire.set_workspace_limit(full + 4096)
        with claire.Registration(shape, nt, w["beta"], w["gamma"]) as reg:
            reg.set_images(m0, m1)
            with pytest.raises(claire.ClaireError) as e:
                reg.mismatch_forward(v, checkpoint_stride=2)
            assert e.value.code == OOM
            assert reg.workspace_bytes() == full  # the failed group was released
            # the context still works, and the differentiable form once the cap is lifted
            _, J = reg.gradient(v)
            assert np.isfinite(J)
            claire.set_workspace_limit(0)
            _, mis = reg.mismatch_forward(v, checkpoint_stride=2)
            _, mis_ref = reg.forward(v)
            torch.cuda.synchronize()
            assert np.isfinite(mis) and abs(mis - mis_ref) <= 1e-6 * abs(mis_ref)
    finally:
        claire.set_workspace_limit(0)
    with claire.Registration(shape, nt, w["beta"], w["gamma"]) as reg:
        assert reg.workspace_bytes() == full


def test_nan_image_reports_nonfinite(claire):
    w, m0, m1 = sin32()
    bad = m0.clone()
    bad[3, 4, 5] = float("nan")
    with claire.Registration(w["shape"], w["nt"], w["beta"], w["gamma"]) as reg:
        reg.set_images(bad, m1)
        v = torch.zeros((3,) + w["shape"], device="cuda")
        rep = reg.solve(v, check=False)
        assert rep.status == NONFINITE and rep.n_gn == 0
        with pytest.raises(claire.ClaireError) as e:
            reg.solve(v)
        assert e.value.code == NONFINITE
        assert float(v.abs().max()) == 0.0  # the initial iterate is kept
        # the same context solves once the images are finite
        reg.set_images(m0, m1)
        rep = reg.solve(v)
        assert rep.status == 0 and rep.n_gn >= 1 and rep.grel <= 5e-2


def test_unreachable_sufficient_decrease_reports_linesearch_failure(claire):
    # J(v + a x) is about J + a s (1 - a/2) along a Gauss-Newton step x with
    # slope s < 0, so c1 = 0.99 needs a <= 0.02; two halvings stop at a = 0.25
    w, m0, m1 = sin32()
    with claire.Registration(w["shape"], w["nt"], w["beta"], w["gamma"]) as reg:
        reg.set_images(m0, m1)
        v = torch.zeros((3,) + w["shape"], device="cuda")
        rep = reg.solve(v, check=False, armijo_c1=0.99, max_ls=2)
        assert rep.status == LINESEARCH and rep.n_gn == 0 and rep.n_ls == 3
        assert float(v.abs().max()) == 0.0  # no step accepted: v is the initial iterate
        assert reg.solve(v).status == 0
