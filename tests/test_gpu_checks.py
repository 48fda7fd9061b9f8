"""The debug build of the library (-DCLAIRE_CHECKS, libclaire_gb_checks.so)
checks every shared-memory box stencil of the transport kernels before its
taps are read: inside the buffer and inside the columns the box copy wrote; a
violation is counted on the device (claire_check_count) and not read.  This
test runs the transport-heavy entry points of the paper's method (gradient,
Hessian matvec, interpolation, a solve) through that build on grids with
ragged tiles, odd sizes, unaligned rows, a mix of box and gather tiles and
large wrapping displacements, and expects zero violations and the release
build's results.  It runs in a child process so that the release library
loaded by the other tests stays untouched."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, json, numpy as np, torch
sys.path.insert(0, ROOT)
from paper_2008_12820_gb300 import build, claire, synth
claire.load(build.build(checks=True))
torch.cuda.set_device(0)
dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
out = {"cases": []}
claire.check_count(reset=True)
cases = [((20, 27, 45), 0.8, 2), ((48, 40, 36), 0.8, 3), ((32, 40, 48), 12.0, 2), ((64, 24, 96), 0.8, 4),
         ((32, 48, 64), "bump", 2), ((128, 128, 128), 0.5, 4)]
for shape, scale, nt in cases:
    d = synth.sinusoid_pair(shape, 1000) if shape[0] != 128 else synth.workload("blob256", shape=shape)
    v = d["v_true"].astype(np.float32)
    if scale == "bump":
        x = np.meshgrid(*synth.grid_axes(shape), indexing="ij")
        bump = np.exp(-((x[0] - 3.0) ** 2 + (x[1] - 2.5) ** 2 + (x[2] - 3.5) ** 2) / 0.15)
        v = (0.5 * v).copy()
        v[2] += (4.0 * bump).astype(np.float32)
        v[1] -= (3.0 * bump).astype(np.float32)
    else:
        v = (scale * v).astype(np.float32)
    vt = synth.smooth_direction(shape, 11)
    with claire.Registration(shape, nt, 1e-2, 1.0) as reg:
        reg.set_images(dev(d["m0"]), dev(d["m1"]))
        g, J = reg.gradient(dev(v))
        H = reg.hess_matvec(None, dev(vt))
        f = reg.interp(dev(d["m0"]), reg.field("dispm"))
        torch.cuda.synchronize()
        out["cases"].append({"shape": list(shape), "J": J, "g": float(g.double().norm()), "H": float(H.double().norm()),
                             "f": float(f.double().norm())})
w = synth.workload("sin32")
with claire.Registration(w["shape"], w["nt"], w["beta"], w["gamma"]) as reg:
    reg.set_images(dev(w["m0"]), dev(w["m1"]))
    v = torch.zeros((3,) + w["shape"], device="cuda")
    rep = reg.solve(v)
    out["solve_J"] = rep.J
out["violations"] = claire.check_count()
print("RESULT " + json.dumps(out))
"""


def run_child(lib_kind):
    code = CHILD.replace("ROOT", repr(ROOT))
    if lib_kind == "release":
        code = code.replace("claire.load(build.build(checks=True))", "claire.load(build.build())")
        code = code.replace('claire.check_count(reset=True)', "")
        code = code.replace('out["violations"] = claire.check_count()', 'out["violations"] = 0')
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=1500, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    import json
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


def test_checked_build_finds_no_box_violation():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    chk = run_child("checks")
    rel = run_child("release")
    assert chk["violations"] == 0
    # the checks change nothing when nothing is violated
    for a, b in zip(chk["cases"], rel["cases"]):
        for k in ("J", "g", "H", "f"):
            assert abs(a[k] - b[k]) <= 1e-6 * abs(b[k]), (a["shape"], k, a[k], b[k])
    assert abs(chk["solve_J"] - rel["solve_J"]) <= 1e-6 * abs(rel["solve_J"])
