"""The batched form (claire_solve_batch): several registrations of uneven
grid sizes solved together, each on a stream and host thread of its own.
Each pair's kernels and their order on its stream are those of a plain
solve, and every reduction has a fixed grid, so the results must equal the
one-by-one solves bit for bit; the oracle pins one pair."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def pairs():
    """uneven grids, time steps, parameters and one FP16-storage context"""
    spec = [((32, 32, 32), 4, 1e-2, "fp32"), ((48, 40, 36), 3, 1e-2, "fp32"),
            ((64, 64, 64), 4, 1e-2, "fp16"), ((40, 48, 60), 2, 5e-2, "fp32"),
            ((96, 96, 96), 4, 1e-2, "fp32"), ((20, 27, 45), 4, 1e-2, "fp32")]
    out = []
    for i, (shape, nt, beta, prec) in enumerate(spec):
        d = synth.blob_pair(shape, 2000 + i, max_disp_vox=2.0)
        out.append(dict(d, shape=shape, nt=nt, beta=beta, gamma=1.0, precision=prec))
    return out


def make(C, w):
    reg = C.Registration(w["shape"], w["nt"], w["beta"], w["gamma"], precision=w["precision"])
    reg.set_images(dev(w["m0"]), dev(w["m1"]))
    return reg


def test_batch_equals_one_by_one(claire):
    ws = pairs()
    seq = []
    for w in ws:
        with make(claire, w) as reg:
            v = torch.zeros((3,) + w["shape"], device="cuda")
            rep = reg.solve(v)
            seq.append((rep, v.clone()))
    regs = [make(claire, w) for w in ws]
    vs = [torch.zeros((3,) + w["shape"], device="cuda") for w in ws]
    reps = claire.solve_batch(regs, vs)
    torch.cuda.synchronize()
    for (r1, v1), r2, v2 in zip(seq, reps, vs):
        assert r2.status == 0 and r2.grel <= 5e-2
        assert (r1.n_gn, r1.n_pcg, r1.n_ls) == (r2.n_gn, r2.n_pcg, r2.n_ls)
        assert r1.J == r2.J and r1.grel == r2.grel
        assert torch.equal(v1, v2)
    # the first pair against the FP64 oracle (1e-4 after a solve)
    w = ws[0]
    P = O.Problem(w["m0"], w["m1"], w["nt"], w["beta"], w["gamma"])
    vo, ro = P.solve(np.zeros((3,) + w["shape"]))
    v0 = vs[0].cpu().numpy().astype(np.float64)
    assert np.linalg.norm(v0 - vo) / np.linalg.norm(vo) < 1e-4
    assert abs(reps[0].J - ro.J) / abs(ro.J) < 1e-4
    for r in regs:
        r.close()


def test_batch_more_pairs_than_workers(claire):
    """Twelve pairs: more than the batch's eight worker threads, so workers
    take several pairs in turn on their stream (largest grid first); every
    result equals the one-by-one solve bit for bit."""
    shapes = [(32, 32, 32), (24, 40, 32), (40, 24, 36), (32, 48, 24), (30, 30, 40), (36, 36, 36),
              (20, 27, 45), (48, 32, 32), (32, 32, 40), (40, 24, 30), (24, 24, 24), (40, 40, 24)]
    ws = []
    for i, shape in enumerate(shapes):
        d = synth.blob_pair(shape, 3000 + i, max_disp_vox=2.0)
        ws.append(dict(d, shape=shape, nt=2 + i % 3, beta=1e-2, gamma=1.0, precision="fp32"))
    seq = []
    for w in ws:
        with make(claire, w) as reg:
            v = torch.zeros((3,) + w["shape"], device="cuda")
            rep = reg.solve(v)
            seq.append((rep, v.clone()))
    regs = [make(claire, w) for w in ws]
    vs = [torch.zeros((3,) + w["shape"], device="cuda") for w in ws]
    reps = claire.solve_batch(regs, vs)
    torch.cuda.synchronize()
    for (r1, v1), r2, v2 in zip(seq, reps, vs):
        assert r2.status == 0
        assert (r1.n_gn, r1.n_pcg, r1.n_ls) == (r2.n_gn, r2.n_pcg, r2.n_ls)
        assert r1.J == r2.J and r1.grel == r2.grel
        assert torch.equal(v1, v2)
    for r in regs:
        r.close()


def test_batch_reports_a_failing_pair(claire):
    ws = pairs()[:3]
    regs = [make(claire, w) for w in ws]
    # the middle pair has no images: it fails with CLAIRE_ERR_STATE, the others solve
    bad = claire.Registration(ws[1]["shape"], ws[1]["nt"], 1e-2, 1.0)
    regs[1].close()
    regs[1] = bad
    vs = [torch.zeros((3,) + w["shape"], device="cuda") for w in ws]
    reps = claire.solve_batch(regs, vs, check=False)
    assert reps[1].status == 4
    assert reps[0].status == 0 and reps[2].status == 0
    with pytest.raises(claire.ClaireError) as e:
        claire.solve_batch(regs, vs)
    assert e.value.code == 4
    for r in regs:
        r.close()


def test_batch_invalid_arguments(claire):
    w = pairs()[0]
    reg = make(claire, w)
    v = torch.zeros((3,) + w["shape"], device="cuda")
    with pytest.raises(claire.ClaireError) as e:   # the same context twice
        claire.solve_batch([reg, reg], [v, v.clone()])
    assert e.value.code == 1
    reg.close()


def test_graph_replayed_matvec_equals_direct_launches(claire):
    """On a stream of its own the solver runs the PCG loop (InvA) and the
    InvH0 inner loop as CUDA graphs with conditional while nodes, and replays
    the captured matvec otherwise; on the legacy stream it launches the
    kernels one by one and decides on the host.  Same arithmetic, same order:
    the solves must agree bit for bit (FP32 and FP16-storage forms, InvA and
    InvH0)."""
    w = pairs()[4]
    for prec, pc in [("fp32", "invA"), ("fp16", "invA"), ("fp32", "invH0")]:
        out = []
        for st in (None, torch.cuda.Stream()):
            with torch.cuda.stream(st) if st is not None else torch.cuda.stream(torch.cuda.default_stream()):
                reg = claire.Registration(w["shape"], w["nt"], w["beta"], w["gamma"], precision=prec)
                reg.set_images(dev(w["m0"]), dev(w["m1"]))
                v = torch.zeros((3,) + w["shape"], device="cuda")
                rep = reg.solve(v, precond=pc)
                torch.cuda.synchronize()
                out.append((rep, v.clone(), reg.launch_count()))
                reg.close()
        (r1, v1, n1), (r2, v2, n2) = out
        assert r1.n_pcg == r2.n_pcg and r1.J == r2.J, (prec, pc)
        assert torch.equal(v1, v2), (prec, pc)
        # replays count the kernels they stand for; the graph path adds its
        # device-side loop-control kernels (and one unused preconditioner
        # application at the end of each loop)
        assert n2 > n1 > 0, (prec, pc, n1, n2)


def test_side_stream_linearization_equals_serial(claire):
    """After an accepted line-search step the solver computes X+, div v and
    the adjoint factor on a second stream beside grad m^j; with the profiler
    on (launches timed one by one) it runs them in order on one stream.  The
    solves must agree bit for bit."""
    w = pairs()[3]
    out = []
    for prof in (False, True):
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            reg = claire.Registration(w["shape"], w["nt"], w["beta"], w["gamma"])
            reg.set_images(dev(w["m0"]), dev(w["m1"]))
            reg.profile_enable(prof)
            v = torch.zeros((3,) + w["shape"], device="cuda")
            rep = reg.solve(v)
            torch.cuda.synchronize()
            out.append((rep.n_gn, rep.n_pcg, rep.J, v.clone()))
            reg.close()
    assert out[0][0] == out[1][0] and out[0][0] >= 2
    assert out[0][1:3] == out[1][1:3]
    assert torch.equal(out[0][3], out[1][3])
