"""The differentiable form: TransportMismatch (torch.autograd.Function) whose
backward is the hand-written adjoint solve plus body force, with the state
checkpointed every k steps (the 256^3 differentiable workload: N_t = 8, k = 2).

Checked against the FP64 oracle (the Euclidean gradient h^3 int lambda grad m
dt of the mismatch, Eq. 3.1 without the regularization term) at 64^3, for
bitwise independence of the checkpoint stride, for an upstream gradient on
m(1), and against central finite differences (h = 1e-3) along five random
smooth directions, at 64^3 (bounded by the oracle's own optimize-then-
discretize gap on the same direction) and at 256^3."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2008_12820_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_12820_gb300 import autograd, claire
    return claire, autograd


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def setup(n, nt=8):
    w = synth.workload("blob256_nt8", shape=(n, n, n))
    v = (0.5 * w["v_true"]).astype(np.float32)
    return w, v


def gpu_grad(C, reg, v, k):
    claire, ag = C
    vv = dev(v).requires_grad_(True)
    mis, m1p = ag.TransportMismatch.apply(vv, reg, k)
    mis.backward()
    torch.cuda.synchronize()
    return float(mis.detach()), vv.grad.detach().cpu().numpy().astype(np.float64)


def test_autograd_matches_oracle_64(C):
    claire, ag = C
    n = 64
    w, v = setup(n)
    P = O.Problem(w["m0"], w["m1"], 8, 1e-2, 1.0)
    g, _ = P.gradient(v)
    b = g - O.apply_A(v, 1e-2, 1.0)
    h3 = (2 * np.pi / n) ** 3
    _, mis_o, _ = P.objective(v)
    with claire.Registration((n, n, n), 8, 1e-2, 1.0) as reg:
        reg.set_images(dev(w["m0"]), dev(w["m1"]))
        mis, gv = gpu_grad(C, reg, v, 2)
    assert abs(mis - mis_o) / mis_o < 1e-5
    assert rel(gv, h3 * b) < 1e-5


def test_checkpoint_stride_does_not_change_the_gradient(C):
    claire, ag = C
    n = 48
    w, v = setup(n)
    out = []
    for k in (1, 2, 3, 8):
        with claire.Registration((n, n, n), 8, 1e-2, 1.0) as reg:
            reg.set_images(dev(w["m0"]), dev(w["m1"]))
            out.append(gpu_grad(C, reg, v, k))
    for mis, gv in out[1:]:
        assert mis == out[0][0]
        assert np.array_equal(gv, out[0][1])


def test_checkpoint_stride_chosen_from_free_memory(C):
    """stride 0: every state kept (stride 1, nothing recomputed) when the
    memory allows; under a workspace cap that leaves room only for a sparser
    set of checkpoints, the stride that needs the least memory; the gradient
    is the same bit for bit either way."""
    claire, ag = C
    n, nt = 48, 8
    w, v = setup(n)
    out = []
    with claire.Registration((n, n, n), nt, 1e-2, 1.0) as reg:
        reg.set_images(dev(w["m0"]), dev(w["m1"]))
        out.append(gpu_grad(C, reg, v, 0))
        assert reg.checkpoint_stride() == 1
    # the differentiable form needs (ceil(nt/k) + 1 + (k + 1 if k > 1) + 8) N
    # floats: 17 N for k = 1, 16 N for k = 2, 3, 4; a cap between the two
    # leaves k = 2 (the first stride of least memory)
    N = n ** 3
    with claire.Registration((n, n, n), nt, 1e-2, 1.0) as reg:
        reg.set_images(dev(w["m0"]), dev(w["m1"]))
        held = reg.workspace_bytes()
        try:
            claire.set_workspace_limit(held + int(16.5 * 4 * N))
            out.append(gpu_grad(C, reg, v, 0))
            assert reg.checkpoint_stride() == 2
        finally:
            claire.set_workspace_limit(0)
    with claire.Registration((n, n, n), nt, 1e-2, 1.0) as reg:
        reg.set_images(dev(w["m0"]), dev(w["m1"]))
        held = reg.workspace_bytes()
        try:
            claire.set_workspace_limit(held + int(15.5 * 4 * N))
            with pytest.raises(claire.ClaireError) as e:
                gpu_grad(C, reg, v, 0)
            assert e.value.code == 2
        finally:
            claire.set_workspace_limit(0)
    assert out[1][0] == out[0][0] and np.array_equal(out[1][1], out[0][1])


def test_upstream_gradient_on_m1(C):
    """loss = mismatch + <w, m(1)>: the adjoint starts from m1 - m(1) - w/h^3."""
    claire, ag = C
    n = 32
    w, v = setup(n)
    rng = np.random.default_rng(0)
    wt = rng.standard_normal((n, n, n)).astype(np.float32) * 1e-3
    P = O.Problem(w["m0"], w["m1"], 8, 1e-2, 1.0)
    P.linearize(v)
    h3 = (2 * np.pi / n) ** 3
    mT = P.state_history()[-1]
    lfinal = (w["m1"].astype(float) - mT) - wt.astype(float) / h3
    lh = O.adjoint(P.dispp(), P.divv(), P.divv_at_xp(), lfinal, 8)
    ref = h3 * O.bodyforce(lh, P.grad_state_history())
    with claire.Registration((n, n, n), 8, 1e-2, 1.0) as reg:
        reg.set_images(dev(w["m0"]), dev(w["m1"]))
        vv = dev(v).requires_grad_(True)
        mis, m1p = ag.transport_mismatch(vv, reg, 2)
        loss = mis + (m1p.double() * dev(wt).double()).sum()
        loss.backward()
        torch.cuda.synchronize()
        assert rel(vv.grad.cpu().numpy(), ref) < 1e-5


def fd_check(C, reg, v, dirs, eps=1e-3):
    claire, ag = C
    _, gv = gpu_grad(C, reg, v, 2)
    gaps = []
    for d in dirs:
        mp = reg.mismatch_forward(dev(v + eps * d), 2)[1]
        mm = reg.mismatch_forward(dev(v - eps * d), 2)[1]
        fd = (mp - mm) / (2 * eps)
        an = float(np.sum(gv * d))
        gaps.append(abs(fd - an) / abs(an))
    return gaps


def test_finite_differences_64_within_oracle_gap(C):
    claire, ag = C
    n = 64
    w, v = setup(n)
    dirs = [synth.smooth_direction((n, n, n), 100 + s) for s in range(5)]
    P = O.Problem(w["m0"], w["m1"], 8, 1e-2, 1.0)
    g, _ = P.gradient(v)
    b = g - O.apply_A(v, 1e-2, 1.0)
    h3 = (2 * np.pi / n) ** 3
    ogaps = []
    for d in dirs:
        fd = (P.objective(v + 1e-3 * d.astype(float))[1] - P.objective(v - 1e-3 * d.astype(float))[1]) / 2e-3
        an = h3 * np.sum(b * d)
        ogaps.append(abs(fd - an) / abs(an))
    with claire.Registration((n, n, n), 8, 1e-2, 1.0) as reg:
        reg.set_images(dev(w["m0"]), dev(w["m1"]))
        gaps = fd_check(C, reg, v, dirs)
    for gg, og in zip(gaps, ogaps):
        assert gg <= 2 * og + 1e-3, (gaps, ogaps)


def test_finite_differences_256(C):
    """the 256^3 differentiable workload (N_t = 8, k = 2) against central
    differences along five smooth directions"""
    claire, ag = C
    n = 256
    w, v = setup(n)
    dirs = [synth.smooth_direction((n, n, n), 200 + s) for s in range(5)]
    with claire.Registration((n, n, n), 8, 1e-2, 1.0) as reg:
        reg.set_images(dev(w["m0"]), dev(w["m1"]))
        gaps = fd_check(C, reg, v, dirs)
    assert max(gaps) < 1e-2, gaps
