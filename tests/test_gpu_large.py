"""The large single pair: 768^3 blob images (60 ellipsoids, sigma 3 voxels),
N_t = 8, stored trajectories in FP16.  A full solve in the FP16-storage form
is compared with the FP32 form at 768^3, and both forms with the FP64 oracle
on the 96^3 spectral restriction of the same images (Fourier truncation to
|k_d| < 48).  The 768^3 images are made on the host, two 768^3 solves hold up
to ~200 GB of HBM one after the other and the 96^3 oracle solve runs on the
host cores (about 2.5 minutes in all on a GB300 node).
Tolerance: 1e-4 after a solve for both forms (the FP16-storage form rounds
only stored copies of FP32 fields, see test_gpu_fp16)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2008_12820_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_SOLVE = 1e-4


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def restrict(f, n):
    """Fourier truncation of a periodic real field to n points per axis
    (wavenumbers |k_d| < n/2; amplitudes kept, so samples scale by 1)."""
    N = f.shape
    F = np.fft.rfftn(f.astype(np.float64))
    h = n // 2
    G = np.zeros((n, n, h + 1), dtype=np.complex128)
    for a in (slice(0, h), slice(-h + 1, None)):
        for b in (slice(0, h), slice(-h + 1, None)):
            G[a, b, :h] = F[a, b, :h]
    scale = (n ** 3) / float(N[0] * N[1] * N[2])
    return (np.fft.irfftn(G * scale, s=(n, n, n), axes=(0, 1, 2))).astype(np.float32)


@pytest.fixture(scope="module")
def claire():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2008_12820_gb300 import claire as C
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return C


def solve(C, w, shape, precision):
    with C.Registration(shape, w["nt"], w["beta"], w["gamma"], precision=precision) as reg:
        reg.set_images(torch.from_numpy(w["m0"]).cuda(), torch.from_numpy(w["m1"]).cuda())
        v = torch.zeros((3,) + tuple(shape), device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        rep = reg.solve(v)
        e1.record()
        torch.cuda.synchronize()
        out = v.cpu().numpy()
        del v
    torch.cuda.empty_cache()
    return rep, out, e0.elapsed_time(e1)


def test_large_pair_fp16_storage(claire):
    w = synth.workload("blob768")
    shape, nt = w["shape"], w["nt"]
    r32, v32, t32 = solve(claire, w, shape, "fp32")
    r16, v16, t16 = solve(claire, w, shape, "fp16")
    print(f"\n768^3 fp32: {r32.n_gn} GN {r32.n_pcg} PCG J {r32.J:.9g} grel {r32.grel:.4g} "
          f"mismatch {r32.mismatch_rel:.6g} {t32:.0f} ms")
    print(f"768^3 fp16: {r16.n_gn} GN {r16.n_pcg} PCG J {r16.J:.9g} grel {r16.grel:.4g} "
          f"mismatch {r16.mismatch_rel:.6g} {t16:.0f} ms; |v16-v32|/|v32| {rel(v16, v32):.3g}")
    assert r32.status == 0 and r16.status == 0
    assert r32.grel <= 5e-2 and r16.grel <= 5e-2
    assert r16.n_gn == r32.n_gn and abs(r16.n_pcg - r32.n_pcg) <= 1
    assert abs(r16.J - r32.J) / abs(r32.J) < TOL_SOLVE
    assert rel(v16, v32) < TOL_SOLVE

    # the 96^3 restriction against the FP64 oracle
    n = 96
    wr = dict(w, m0=restrict(w["m0"], n), m1=restrict(w["m1"], n))
    P = O.Problem(wr["m0"], wr["m1"], nt, w["beta"], w["gamma"])
    vo, ro = P.solve(np.zeros((3, n, n, n)))
    q32, u32, _ = solve(claire, wr, (n, n, n), "fp32")
    q16, u16, _ = solve(claire, wr, (n, n, n), "fp16")
    print(f"96^3 restriction: oracle J {ro.J:.9g} ({ro.n_gn} GN {ro.n_pcg} PCG); "
          f"fp32 rel v {rel(u32, vo):.3g} J {abs(q32.J - ro.J) / abs(ro.J):.3g}; "
          f"fp16 rel v {rel(u16, vo):.3g} J {abs(q16.J - ro.J) / abs(ro.J):.3g}")
    assert q32.n_gn == ro.n_gn and q16.n_gn == ro.n_gn
    assert rel(u32, vo) < TOL_SOLVE and abs(q32.J - ro.J) / abs(ro.J) < TOL_SOLVE
    assert rel(u16, vo) < TOL_SOLVE and abs(q16.J - ro.J) / abs(ro.J) < TOL_SOLVE
