"""claire_solve_host: set_images + solve with host buffers, the copies
overlapped with the computation, gives the device solve's results bit for
bit (FP32 and FP16-storage forms, page-locked and pageable buffers, input and
output aliased or not, a solve that accepts no step)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2008_12820_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def claire():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2008_12820_gb300 import claire as C
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return C


def device_solve(C, w, shape, precision, v0, **opts):
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream), C.Registration(shape, w["nt"], w["beta"], w["gamma"], stream=stream,
                                                   precision=precision) as reg:
        reg.set_images(torch.from_numpy(w["m0"]).cuda(), torch.from_numpy(w["m1"]).cuda())
        v = torch.from_numpy(v0.copy()).cuda()
        rep = reg.solve(v, **opts)
        torch.cuda.synchronize()
        return rep, v.cpu().numpy()


@pytest.mark.parametrize("precision,pin,alias", [("fp32", True, False), ("fp32", False, True),
                                                 ("fp16", True, True)])
def test_host_solve_equals_device_solve(claire, precision, pin, alias):
    w = synth.workload("blob256", shape=(64, 64, 64))
    shape = w["shape"]
    v0 = np.zeros((3,) + shape, dtype=np.float32)
    r_dev, v_dev = device_solve(claire, w, shape, precision, v0)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream), claire.Registration(shape, w["nt"], w["beta"], w["gamma"], stream=stream,
                                                        precision=precision) as reg:
        m0, m1 = torch.from_numpy(w["m0"]), torch.from_numpy(w["m1"])
        vin = torch.from_numpy(v0.copy())
        if pin:
            m0, m1, vin = m0.pin_memory(), m1.pin_memory(), vin.pin_memory()
        vout = vin if alias else (torch.empty_like(vin).pin_memory() if pin else torch.empty_like(vin))
        # run twice: the second call reuses the context's device copy of v
        for _ in range(2):
            if alias:
                vin.zero_()
            rep = reg.solve_host(m0, m1, vin, vout)
            assert rep.status == 0
            assert np.array_equal(vout.numpy(), v_dev)
            assert rep.J == r_dev.J and rep.g == r_dev.g
            assert (rep.n_gn, rep.n_pcg, rep.n_ls) == (r_dev.n_gn, r_dev.n_pcg, r_dev.n_ls)
        # the images stay set for the device-side API
        g = torch.empty((3,) + shape, device="cuda")
        reg.gradient(torch.from_numpy(v_dev).cuda(), out=g)
        torch.cuda.synchronize()
        assert torch.isfinite(g).all()


def test_host_solve_without_accepted_step(claire):
    """max_gn = 0: no step; the initial velocity comes back unchanged"""
    w = synth.workload("sin32")
    shape = w["shape"]
    v0 = (0.3 * synth.smooth_direction(shape, 5)).astype(np.float32)
    with claire.Registration(shape, w["nt"], w["beta"], w["gamma"]) as reg:
        vin = torch.from_numpy(v0.copy()).pin_memory()
        vout = torch.full_like(vin, 7.0).pin_memory()
        rep = reg.solve_host(torch.from_numpy(w["m0"]), torch.from_numpy(w["m1"]), vin, vout, max_gn=0)
        assert rep.n_gn == 0
        assert np.array_equal(vout.numpy(), v0)


def test_host_solve_rejects_device_tensors(claire):
    w = synth.workload("sin32")
    shape = w["shape"]
    with claire.Registration(shape, w["nt"], w["beta"], w["gamma"]) as reg:
        with pytest.raises(ValueError):
            reg.solve_host(torch.from_numpy(w["m0"]).cuda(), torch.from_numpy(w["m1"]),
                           torch.zeros((3,) + shape))
        with pytest.raises(ValueError):
            reg.solve_host(torch.from_numpy(w["m0"]), torch.from_numpy(w["m1"]), torch.zeros((3, 4, 4, 4)))
