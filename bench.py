#!/usr/bin/env python
"""Benchmark of the GB300 registration hot path.

One step = one full Gauss-Newton-Krylov solve (Algorithm 1 of arXiv
2008.12820) of the 256^3 synthetic blob workload: N_t = 4, beta = 1e-2,
gamma = 1, inverse-A preconditioner, stop at 5e-2 relative gradient
reduction, started from v = 0.  Every row of the hot path runs inside it:
RK2 foot points, cubic interpolation, state / adjoint / incremental transport,
spectral gradient / divergence / regularization / preconditioner, PCG with FP64
dots, Armijo line search.  The inputs are resident in HBM before the timed
region; the working set (~5 GB) is far larger than the 129 MB L2.

value = voxels registered per second (N / solve time, Gvoxel/s), summed over
ranks.  With torchrun (N > 1) every rank solves its own replica (no
collective on the data path; "replicas only").

Extra keys: Hessian-matvec throughput, the solve report, a roofline entry for
the dominant kernel class (algorithmic bytes / CUDA-event time, live), an
end-to-end number through the C ABI with host buffers, a CPU baseline of the
FP64 oracle, the error against the oracle, clocks sampled during the timed
region.

``--impl reference`` times the FP64 CPU oracle (the only reference this
method has; the paper's code is not available) on the same metric.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("Hessian matvec Gvoxel/s and GN solve time @256³; % of HBM roofline; "
          "err vs FP64")
UNIT = "Gvoxel/s"
WORKLOAD = "blob256"
WORKLOAD_DESCS = {
    "blob256": ("256^3 synthetic brain-like blob images (12 ellipsoids, sigma 2 voxels), "
                "reference warped by a band-limited displacement (|k|<=6, max 4 voxels); "
                "nt=4, beta=1e-2, gamma=1, cubic SL, spectral ops, PC InvA, "
                "full GN-Krylov solve to 5e-2 from v=0"),
    "blob768": ("768^3 synthetic brain-like blob images (60 ellipsoids, sigma 3 voxels), "
                "reference warped by a band-limited displacement (|k|<=6, max 4 voxels); "
                "nt=8, beta=1e-2, gamma=1, cubic SL, spectral ops, PC InvA, "
                "full GN-Krylov solve to 5e-2 from v=0"),
}
WORKLOAD_DESC = WORKLOAD_DESCS[WORKLOAD]
CPU_SAMPLE_N = 64        # oracle solves the same generator on a 64^3 grid
ERR_CHECK_N = 128        # GPU vs oracle gradient / matvec on a 128^3 instance

KCLASS = ["footpoint", "state", "adjoint", "incstate", "incadj", "bodyforce", "fft_r2c",
          "fft_c2c", "fft_mul", "fft_c2r", "reduce", "vector", "interp", "fd", "deriv"]
# kernel function names of each class (for the ncu summaries); the template
# argument of k_sl_pipe is the step kind: 0 plain, 1 adjoint, 2 incremental
# state, 3 adjoint factor, 4 last incremental-state step, 5 adjoint step that
# adds its body-force term, 6 the same with the curvature dot
KNAMES = {"footpoint": "k_footpoints_box, k_footpoints, k_tile_ranges, k_sl_pipe<3, *>",
          "state": "k_sl_pipe<0, *>", "adjoint": "k_sl_pipe<5, *>", "incstate": "k_sl_pipe<2, *>, k_sl_pipe<4, *>",
          "incadj": "k_sl_pipe<5, *>, k_sl_pipe<6, *>", "bodyforce": "k_adjfinal_acc",
          "fft_r2c": "k_r2c_x3_p (k_r2c_x3 for unaligned rows)", "fft_c2c": "k_c2c_x2", "fft_mul": "k_mul_x1",
          "fft_c2r": "k_c2r_x3_p (k_c2r_x3 for unaligned spectra)",
          "reduce": "k_reduce2, k_stats, k_finalize, k_finalize4",
          "vector": "k_pcg_update, k_pcg_dir_u0, k_axpby, k_incstate_init, k_f2h, k_h2f",
          "interp": "k_sl_pipe<0, *>", "fd": "k_grad_fd8, k_div_fd8",
          "deriv": "k_deriv_x3_p, k_deriv_strided_p (k_deriv_x3, k_deriv_strided for unaligned rows)"}


# the transport and transform classes (every one of them is asked to reach
# 60% of the HBM peak); the others are streaming vector work and reductions
TRANSPORT_FFT = ("footpoint", "state", "adjoint", "incstate", "incadj", "fft_r2c", "fft_c2c", "fft_mul",
                 "fft_c2r", "deriv")
# one cubic SL interpolation per voxel and launch (the bench's solves use cubic interpolation)
SL_STEP_CLASSES = ("state", "adjoint", "incstate", "incadj")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16"],
                    help="fp16: stored state / adjoint trajectories in FP16 (FP32 arithmetic)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the InvH0 / 2LInvH0 solves and the batched form in the default line")
    ap.add_argument("--no-fft-reference", action="store_true",
                    help="skip the cuFFT reference point (profiling captures of the library's kernels)")
    ap.add_argument("--grid", type=int, default=0,
                    help="run the same generator on an n^3 grid (profiling captures; not a bench line)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate_ranks(ms_local, n_vox_local, world_size, device=None):
    """Job-level numbers of the replica run: the slowest rank's time per step
    (max over ranks) and the voxels all ranks registered per second.  Each rank
    solves its own registration, so the only collective is this reduction."""
    import torch
    if world_size > 1:
        import torch.distributed as dist
        t = torch.tensor([float(ms_local), float(n_vox_local)], dtype=torch.float64,
                         device=device)
        mx = t.clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        tot = t.clone()
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
        ms, vox = float(mx[0].item()), float(tot[1].item())
    else:
        ms, vox = float(ms_local), float(n_vox_local)
    return ms, vox / (ms * 1e-3) / 1e9


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.gpu = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = max(smax, float(r[2]))
                for nm, val in zip(names, r[5:9]):
                    if val.strip().lower() in ("active", "1", "yes"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def traffic_for(kclass, bytes_per_launch, n_vox):
    """DRAM traffic per launch from the committed ncu summary of this kernel,
    scaled by voxels; null if the kernel source changed since the capture."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(kclass)
    if not e:
        return None
    src = os.path.join(ROOT, e["source"])
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] if os.path.exists(src) else None
    if h != e.get("source_sha256_16"):
        return None
    return e["dram_bytes_per_voxel"] * n_vox * e.get("voxels_per_launch_factor", 1.0)


# ---------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    import __graft_entry__
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    __graft_entry__.build()
    from paper_2008_12820_gb300 import claire, synth

    w = synth.workload(args.workload, shape=(args.grid,) * 3 if args.grid else None)
    shape, nt, beta, gamma = w["shape"], w["nt"], w["beta"], w["gamma"]
    N = int(np.prod(shape))
    # a stream of its own (not the legacy default stream), so that the library
    # can capture the PCG matvec into a CUDA graph
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    m0 = torch.from_numpy(w["m0"]).cuda()
    m1 = torch.from_numpy(w["m1"]).cuda()
    v = torch.zeros((3,) + shape, device="cuda")
    reg = claire.Registration(shape, nt, beta, gamma, precision=args.precision)
    reg.set_images(m0, m1)

    def step():
        v.zero_()
        return reg.solve(v)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        rep = step()
    torch.cuda.synchronize()

    # ---- timed region ----------------------------------------------------
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = reg.launch_count()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    reports = []
    for _ in range(args.steps):
        reports.append(step())
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = reg.launch_count() - launches0
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    ms, value = aggregate_ranks(ms, N, ws, device="cuda")
    rep = reports[-1]

    # ---- per-class kernel times: one more solve with the profiler on (its
    # per-launch events keep the matvec out of the CUDA graph) -------------
    reg.profile_enable(True)
    rep_prof = step()
    torch.cuda.synchronize()
    prof = {k: reg.profile_read(i) for i, k in enumerate(KCLASS)}
    reg.profile_enable(False)

    # ---- Hessian matvec throughput at the solution (own events loop) -------
    reg.linearize(v)
    vt = torch.from_numpy(synth.smooth_direction(shape, 7)).cuda()
    Hv = torch.empty_like(vt)
    for _ in range(3):
        reg.hess_matvec(None, vt, out=Hv)
    torch.cuda.synchronize()
    nmv = 20
    e0.record(stream)
    for _ in range(nmv):
        reg.hess_matvec(None, vt, out=Hv)
    e1.record(stream)
    torch.cuda.synchronize()
    mv_ms = e0.elapsed_time(e1) / nmv
    mv_gvox = N / (mv_ms * 1e-3) / 1e9

    fft_ref = fft_reference(reg, vt, beta, gamma, stream) if rank == 0 and not args.no_fft_reference else None

    # ---- roofline of the dominant kernel class ----------------------------
    peak, peak_src = read_peaks()
    dom = max(prof, key=lambda k: prof[k][1])
    nl, kms, kby = prof[dom]
    achieved = (kby / nl) / ((kms / nl) * 1e-3) / 1e9 if nl else 0.0
    breakdown = {k: {"launches": n_, "ms_per_step": round(t_, 4),
                     "GBps": round(b_ / (t_ * 1e-3) / 1e9, 1) if t_ > 0 else None,
                     "frac": round(b_ / (t_ * 1e-3) / 1e9 / peak, 4) if t_ > 0 else None}
                 for k, (n_, t_, b_) in prof.items() if n_}
    # The SL step classes are bound by the shared-memory data pipe, not by HBM:
    # each voxel of a step reads its 64 cubic stencil taps there, one 128-byte
    # wavefront per warp and tap, so a step over N voxels needs at least
    # 64 N / 32 wavefront-cycles spread over the SMs.  That bound at the SM
    # clock sampled during the timed region, and the class's fraction of it.
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    f_sm = (clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0) * 1e6 if isinstance(clk, dict) else 2070e6
    for k in SL_STEP_CLASSES:
        e = breakdown.get(k)
        if e and e["ms_per_step"] > 0:
            bound_ms = e["launches"] * N * 64 / 32 / sms / f_sm * 1e3
            e["smem_pipe"] = {"bound_ms": round(bound_ms, 4), "frac": round(bound_ms / e["ms_per_step"], 4)}
    tf = {k: e["frac"] for k, e in breakdown.items() if k in TRANSPORT_FFT and e["frac"] is not None}
    min_tf = min(tf, key=tf.get) if tf else None
    roofline = {"bound": "hbm", "kernel": dom, "kernels": KNAMES[dom],
                "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_source": peak_src,
                "traffic": traffic_for(dom, kby / nl if nl else 0, N),
                "bytes_per_launch": kby / nl if nl else 0}

    out = {
        "metric": METRIC, "value": round(value, 5), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_DESCS.get(args.workload, args.workload), "grid": list(shape),
                   "nt": nt, "beta": beta, "gamma": gamma, "precond": "InvA", "eps_n": 5e-2,
                   "storage": "fp16 trajectories" if args.precision == "fp16" else "fp32",
                   "l2": f"inputs larger than L2 (working set {reg.workspace_bytes() / 1e9:.1f} GB)",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "gn_solve_time_s": round(ms * 1e-3, 5),
        "hess_matvec_gvoxel_s": round(mv_gvox, 4), "hess_matvec_ms": round(mv_ms, 4),
        "solve": {"n_gn": rep.n_gn, "n_pcg": rep.n_pcg, "n_matvec": rep.n_matvec,
                  "n_ls": rep.n_ls, "grel": rep.grel, "mismatch_rel": rep.mismatch_rel,
                  "J": rep.J, "t_pcg_ms": round(rep.t_pcg_ms, 3),
                  "phases_of_profiled_solve_ms": {"hess": round(rep_prof.t_hess_ms, 3),
                                                  "grad": round(rep_prof.t_grad_ms, 3),
                                                  "pc": round(rep_prof.t_pc_ms, 3),
                                                  "obj": round(rep_prof.t_obj_ms, 3)},
                  # the Gauss-Newton matvec as the solver applies it inside PCG,
                  # beta A p carried by the recurrence instead of a transform
                  # (events around each launch group: a slight overestimate)
                  "pcg_matvec_ms_profiled": round(rep_prof.t_hess_ms / rep_prof.n_matvec, 4)
                  if rep_prof.n_matvec else None},
        "roofline": roofline, "kernel_breakdown": breakdown,
        "min_frac_transport_fft": {"class": min_tf, "frac": tf.get(min_tf)} if min_tf else None,
        "gpu_launches": int(launches), "clocks": clk,
    }
    if fft_ref is not None:
        out["fft_reference"] = fft_ref

    # ---- end to end through the C ABI with host buffers --------------------
    # claire_solve_host: images and initial v from page-locked host memory,
    # the result back to host memory, the copies overlapped with the solve
    # (each accepted iterate is copied out while the next gradient runs, so
    # the device-to-host bytes are one velocity per accepted step)
    if not args.no_e2e:
        hm0 = torch.from_numpy(w["m0"]).pin_memory()
        hm1 = torch.from_numpy(w["m1"]).pin_memory()
        hv0 = torch.zeros((3,) + shape).pin_memory()
        hv = torch.empty((3,) + shape).pin_memory()

        def e2e_step():
            return reg.solve_host(hm0, hm1, hv0, hv)

        e2e_step()
        torch.cuda.synchronize()
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            r_e = e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        e_ms = e0.elapsed_time(e1) / args.steps
        out["e2e"] = {"value": round(ws * N / (e_ms * 1e-3) / 1e9, 5), "unit": UNIT,
                      "ms_per_step": round(e_ms, 3), "h2d_bytes_per_step": 5 * 4 * N,
                      "d2h_bytes_per_step": 3 * 4 * N * max(1, r_e.n_gn),
                      "api": "claire_solve_host (copies overlapped with the solve)"}

    # ---- the same solve with the paper's H0-based preconditioners ---------
    if not args.no_extra:
        out["precond_solves"] = precond_solves(reg, v, stream)
        out["paper_gpu_discretization"] = paper_gpu_discretization(reg, v, shape, stream)
        if args.workload == "blob256":
            out["large_displacement"] = large_displacement(claire, synth, args, stream)

    # ---- CPU baseline (FP64 oracle) and error vs FP64, rank 0 at N = 1 ------
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        err, t_or = error_vs_oracle(claire, synth, args.precision)
        out["cpu_baseline"] = cpu_baseline_sample()
        out["cpu_baseline"].update(t_or)
        out["err_vs_fp64"] = err
    reg.close()
    # ---- the batched form (16 pairs of uneven grids), rank 0 at N = 1 ------
    if rank == 0 and ws == 1 and not args.no_extra:
        b = run_batch(args, as_extra=True)
        out["batch16"] = {k: b[k] for k in ("value", "unit", "ms_per_step", "one_by_one", "batch_speedup",
                                            "same_results_as_one_by_one", "gpu_launches")}
        out["batch16"]["config"] = b["config"]["workload"]
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def precond_solves(reg, v, stream, reps=3):
    """The benchmark's solve with the InvH0 and two-level InvH0 preconditioners
    (Section 3 "Preconditioning", Algorithm 2; inner tolerance 1e-3 times the
    forcing term): device time per solve, PCG and inner iteration counts."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    for name in ("invH0", "2LinvH0"):
        v.zero_()
        reg.solve(v, precond=name)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            v.zero_()
            rep = reg.solve(v, precond=name)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"solve_ms": round(ms, 3), "n_gn": rep.n_gn, "n_pcg": rep.n_pcg, "n_inner": rep.n_inner,
                     "grel": rep.grel, "J": rep.J, "t_pc_ms": round(rep.t_pc_ms, 3),
                     "t_hess_ms": round(rep.t_hess_ms, 3)}
    return out


def paper_gpu_discretization(reg, v, shape, stream, reps=3):
    """The same solve and Hessian matvec with the discretization the paper's
    GPU runs use (Sections 4.1, 4.2: trilinear SL interpolation, 8th-order
    finite-difference first derivatives), beside the default cubic / spectral
    form; the context is set back to cubic / spectral afterwards."""
    import torch
    from paper_2008_12820_gb300 import synth
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reg.set_discretization(interp="linear", deriv="fd8")
    try:
        v.zero_()
        reg.solve(v)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            v.zero_()
            rep = reg.solve(v)
        e1.record(stream)
        torch.cuda.synchronize()
        solve_ms = e0.elapsed_time(e1) / reps
        reg.linearize(v)
        vt = torch.from_numpy(synth.smooth_direction(shape, 7)).cuda()
        Hv = torch.empty_like(vt)
        for _ in range(3):
            reg.hess_matvec(None, vt, out=Hv)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(10):
            reg.hess_matvec(None, vt, out=Hv)
        e1.record(stream)
        torch.cuda.synchronize()
        mv_ms = e0.elapsed_time(e1) / 10
    finally:
        reg.set_discretization(interp="cubic", deriv="spectral")
    return {"interp": "trilinear", "deriv": "fd8", "solve_ms": round(solve_ms, 3), "n_gn": rep.n_gn,
            "n_pcg": rep.n_pcg, "grel": rep.grel, "J": rep.J, "hess_matvec_ms": round(mv_ms, 4)}


def large_displacement(claire, synth, args, stream, reps=3):
    """The same generator with three times the displacement (12 voxels at
    most, up to 3 cells per time step): solve time and Hessian matvec at the
    solution, beside the default workload's."""
    import torch
    w = synth.workload("blob256_d12")
    shape = w["shape"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with claire.Registration(shape, w["nt"], w["beta"], w["gamma"], precision=args.precision) as reg:
        reg.set_images(torch.from_numpy(w["m0"]).cuda(), torch.from_numpy(w["m1"]).cuda())
        v = torch.zeros((3,) + shape, device="cuda")
        reg.solve(v)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            v.zero_()
            rep = reg.solve(v)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        reg.linearize(v)
        vt = torch.from_numpy(synth.smooth_direction(shape, 7)).cuda()
        Hv = torch.empty_like(vt)
        for _ in range(3):
            reg.hess_matvec(None, vt, out=Hv)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(20):
            reg.hess_matvec(None, vt, out=Hv)
        e1.record(stream)
        torch.cuda.synchronize()
        mv = e0.elapsed_time(e1) / 20
        vmax = float(torch.linalg.vector_norm(v, dim=0).max()) * shape[0] / (2 * 3.141592653589793)
    return {"workload": "blob256 generator with max displacement 12 voxels (seed 1001)", "solve_ms": round(ms, 3),
            "n_gn": rep.n_gn, "n_pcg": rep.n_pcg, "grel": rep.grel, "hess_matvec_ms": round(mv, 4),
            "max_displacement_vox_of_solution": round(vmax, 2)}


def fft_reference(reg, r, beta, gamma, stream, reps=20):
    """cuFFT (through torch.fft) beside the library's own pencil FFT, as a
    reference point only: the library's (beta A)^-1 of a 3-component field
    (forward R2C transforms, the per-wavenumber multiplier, inverse C2R
    transforms) against cuFFT's 3D R2C + C2R of the same three components
    with and without the same multiplier applied by torch elementwise ops.
    Nothing here is on the library's path."""
    import torch
    shape = tuple(r.shape[1:])
    n1, n2, n3 = shape
    s = torch.empty_like(r)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ours_ms = timed(lambda: reg.precond(r, out=s))

    # (beta A)^-1 symbol on the half spectrum: k != 0:
    # (beta|k|^2)^-1 [I - gamma kh kh^T / (beta|k|^2 + gamma|kh|^2)], identity at k = 0;
    # kh is k with the Nyquist index of an even axis set to 0, |k|^2 keeps it
    def wn(n, half=False):
        k = torch.fft.rfftfreq(n, 1.0 / n) if half else torch.fft.fftfreq(n, 1.0 / n)
        kh = k.clone()
        if n % 2 == 0:
            kh[k.abs() == n // 2] = 0.0
        return k.cuda(), kh.cuda()
    (k1, kh1), (k2, kh2), (k3, kh3) = wn(n1), wn(n2), wn(n3, True)
    K = [k1[:, None, None], k2[None, :, None], k3[None, None, :]]
    KH = [kh1[:, None, None].expand(-1, n2, n3 // 2 + 1), kh2[None, :, None].expand(n1, -1, n3 // 2 + 1),
          kh3[None, None, :].expand(n1, n2, -1)]
    k2s = K[0] ** 2 + K[1] ** 2 + K[2] ** 2
    kh2s = KH[0] ** 2 + KH[1] ** 2 + KH[2] ** 2
    zero = k2s == 0
    inv = torch.where(zero, torch.ones_like(k2s), 1.0 / (beta * torch.where(zero, torch.ones_like(k2s), k2s)))
    coup = torch.where(zero, torch.zeros_like(k2s), gamma / (beta * k2s + gamma * kh2s))

    def cufft_mul():
        R = torch.fft.rfftn(r, dim=(1, 2, 3))
        proj = KH[0] * R[0] + KH[1] * R[1] + KH[2] * R[2]
        S = torch.stack([inv * (R[c] - coup * KH[c] * proj) for c in range(3)])
        return torch.fft.irfftn(S, s=shape, dim=(1, 2, 3))

    cufft_ms = timed(lambda: torch.fft.irfftn(torch.fft.rfftn(r, dim=(1, 2, 3)), s=shape, dim=(1, 2, 3)))
    cufft_mul_ms = timed(cufft_mul)
    s_ref = cufft_mul()
    diff = float(torch.linalg.vector_norm(s - s_ref) / torch.linalg.vector_norm(s_ref))
    return {"what": "(beta A)^-1 of a 3-component field: own pencil FFT (R2C, multiplier fused "
                    "into the x1 pass, C2R) vs cuFFT via torch.fft (reference point only)",
            "grid": list(shape), "own_precond_ms": round(ours_ms, 4),
            "cufft_r2c_c2r_3comp_ms": round(cufft_ms, 4),
            "cufft_r2c_mul_c2r_3comp_ms": round(cufft_mul_ms, 4),
            "rel_diff_own_vs_cufft": diff}


def cpu_baseline_sample(steps=1):
    """Time the FP64 oracle's full solve of the same generator on a 64^3 grid
    (host cores, OpenMP over all of them).  Reported per voxel, like value."""
    import numpy as np

    import oracle
    from paper_2008_12820_gb300 import synth
    oracle.build()
    n = CPU_SAMPLE_N
    w = synth.workload(WORKLOAD, shape=(n, n, n))
    P = oracle.Problem(w["m0"], w["m1"], w["nt"], w["beta"], w["gamma"])
    times = []
    for _ in range(steps):
        t = time.perf_counter()
        _, rep = P.solve(np.zeros((3, n, n, n)))
        times.append(time.perf_counter() - t)
    t = min(times)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": round(n ** 3 / t / 1e9, 7), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"full FP64 GN-Krylov solve of the same blob generator on a {n}^3 grid "
                      f"({rep.n_gn} GN, {rep.n_pcg} PCG), {t:.2f} s; voxels/s",
            "seconds": round(t, 3)}


def error_vs_oracle(claire, synth, precision="fp32"):
    """Relative L2 error of the GPU gradient, objective and Hessian matvec
    against the FP64 oracle on the 128^3 instance of the same generator."""
    import numpy as np
    import torch

    import oracle
    n = ERR_CHECK_N
    w = synth.workload(WORKLOAD, shape=(n, n, n))
    v = (0.5 * w["v_true"]).astype(np.float32)
    vt = synth.smooth_direction((n, n, n), 7)
    P = oracle.Problem(w["m0"], w["m1"], w["nt"], w["beta"], w["gamma"])
    t0 = time.perf_counter()
    go, Jo = P.gradient(v)
    t1 = time.perf_counter()
    Ho = P.matvec(vt)
    t2 = time.perf_counter()
    t_or = {"oracle_gradient_s_128": round(t1 - t0, 3), "oracle_matvec_s_128": round(t2 - t1, 3),
            "oracle_matvec_gvoxel_s_128": round(n ** 3 / (t2 - t1) / 1e9, 6)}
    with claire.Registration((n, n, n), w["nt"], w["beta"], w["gamma"], precision=precision) as reg:
        reg.set_images(torch.from_numpy(w["m0"]).cuda(), torch.from_numpy(w["m1"]).cuda())
        g, J = reg.gradient(torch.from_numpy(v).cuda())
        H = reg.hess_matvec(None, torch.from_numpy(vt).cuda())
        torch.cuda.synchronize()
        g, H = g.cpu().numpy().astype(np.float64), H.cpu().numpy().astype(np.float64)

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    def rel_hm1(a, b):
        # relative error in the H^{-1} norm: spectrum weighted by 1/(1 + |k|^2)
        k = [np.fft.fftfreq(n, 1.0 / n)] * 3
        K2 = k[0][:, None, None] ** 2 + k[1][None, :, None] ** 2 + k[2][None, None, :] ** 2
        wgt = 1.0 / (1.0 + K2)
        ea = sum(float(np.sum(np.abs(np.fft.fftn(a[c] - b[c])) ** 2 * wgt)) for c in range(3))
        eb = sum(float(np.sum(np.abs(np.fft.fftn(b[c])) ** 2 * wgt)) for c in range(3))
        return (ea / eb) ** 0.5

    return ({"grid": [n, n, n], "storage": precision, "gradient": rel(g, go), "hess_matvec": rel(H, Ho),
             "objective": abs(J - Jo) / abs(Jo), "gradient_Hm1": rel_hm1(g, go),
             "hess_matvec_Hm1": rel_hm1(H, Ho),
             "note": "L2 errors of fields containing beta*A of a smooth field sit at the FP32 "
                     "noise floor of the forward FFT amplified by |k|^2; H^-1 norm alongside"}, t_or)


# ---------------------------------------------------------------------------
def run_reference(args):
    """The oracle as the reference arm: each step is a full FP64 solve of the
    same generator on a 64^3 grid (a bounded sample of the 256^3 workload)."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_2008_12820_gb300 import synth
    oracle.build()
    n = CPU_SAMPLE_N
    w = synth.workload(WORKLOAD, shape=(n, n, n))
    P = oracle.Problem(w["m0"], w["m1"], w["nt"], w["beta"], w["gamma"])
    for _ in range(args.warmup):
        P.solve(np.zeros((3, n, n, n)))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _, rep = P.solve(np.zeros((3, n, n, n)))
    t = (time.perf_counter() - t0) / args.steps
    value = n ** 3 / t / 1e9
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out = {
        "impl": "reference", "metric": METRIC, "value": round(value, 7), "unit": UNIT,
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(t * 1e3, 2), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "grid": [n, n, n], "sample_of_grid": [256, 256, 256], "nt": 4,
                   "beta": 1e-2, "gamma": 1.0, "precond": "InvA", "eps_n": 5e-2, "storage": "fp64",
                   "parallelism": f"host cores ({cores} OpenMP threads)"},
        "cpu_baseline": {"value": round(value, 7), "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"full FP64 GN-Krylov solve of the same generator on a "
                                   f"{n}^3 grid ({rep.n_gn} GN, {rep.n_pcg} PCG); voxels/s"},
        "e2e": {"value": round(value, 7), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def run_batch(args, as_extra=False):
    """The batched form: 16 blob pairs on grids drawn from {64, 96, 128, 160}^3
    solved together (claire_solve_batch: a stream and host thread per pair)
    against the same 16 solved one by one; one step = all 16 solves.  With
    as_extra the result is returned (a key of the default line) instead of
    printed."""
    import numpy as np
    import torch

    import __graft_entry__
    if not as_extra:
        torch.cuda.set_device(0)
    __graft_entry__.build()
    from paper_2008_12820_gb300 import claire, synth

    ws = synth.batch_workload()
    # a stream of its own for the one-by-one solves, so both arms replay the
    # captured PCG matvec (the batch makes a stream per pair)
    torch.cuda.set_stream(torch.cuda.Stream())
    regs, vs = [], []
    for w in ws:
        r = claire.Registration(w["shape"], w["nt"], w["beta"], w["gamma"])
        r.set_images(torch.from_numpy(w["m0"]).cuda(), torch.from_numpy(w["m1"]).cuda())
        regs.append(r)
        vs.append(torch.zeros((3,) + w["shape"], device="cuda"))
    nvox = sum(int(np.prod(w["shape"])) for w in ws)
    stream = torch.cuda.current_stream()

    def batch_step():
        for v in vs:
            v.zero_()
        return claire.solve_batch(regs, vs)

    def seq_step():
        out = []
        for r, v in zip(regs, vs):
            v.zero_()
            out.append(r.solve(v))
        return out

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            reps = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps, reps

    clocks = ClockSampler(torch.cuda.current_device())
    if not as_extra:
        clocks.start()
    launches0 = sum(r.launch_count() for r in regs)
    ms_b, reps_b = timed(batch_step)
    launches = (sum(r.launch_count() for r in regs) - launches0) // (args.steps + args.warmup)
    clk = clocks.stop() if not as_extra else None
    ms_s, reps_s = timed(seq_step)
    same = all(a.n_pcg == b.n_pcg and a.J == b.J for a, b in zip(reps_b, reps_s))
    sizes = sorted({w["shape"][0] for w in ws})
    out = {
        "metric": "batched GN-Krylov solves Gvoxel/s (16 pairs, uneven grids)", "value": round(nvox / (ms_b * 1e-3) / 1e9, 5),
        "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_b, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "16 blob pairs (12 ellipsoids, sigma 2 voxels, max displacement 4 voxels), grids "
                               f"drawn from {sizes}^3 (seed 1003): "
                               + ", ".join(str(w["shape"][0]) for w in ws)
                               + "; nt=4, beta=1e-2, gamma=1, InvA, each solved to 5e-2 from v=0",
                   "voxels": nvox, "parallelism": "one stream and host thread per pair"},
        "one_by_one": {"value": round(nvox / (ms_s * 1e-3) / 1e9, 5), "ms_per_step": round(ms_s, 3)},
        "batch_speedup": round(ms_s / ms_b, 3), "same_results_as_one_by_one": same,
        "solves": [{"n": w["shape"][0], "n_gn": r.n_gn, "n_pcg": r.n_pcg, "grel": r.grel}
                   for w, r in zip(ws, reps_b)],
        "gpu_launches": int(launches), "clocks": clk,
    }
    for r in regs:
        r.close()
    if as_extra:
        return out
    print(json.dumps(out), flush=True)


def run_pcstudy(args):
    """The preconditioner study of Section 3 ("Preconditioning", Algorithm 2)
    on the synthetic blob pairs: PCG iterations, inner iterations and solve
    time of InvA, InvH0 and two-level InvH0 for beta in {5e-1, 1e-1, 5e-2} at
    128^3 and 256^3 (N_t = 4, gamma = 1, from v = 0 to 5e-2 gradient
    reduction; inner tolerance 1e-3 times the forcing term).  One untimed and
    one timed solve per case."""
    import torch

    import __graft_entry__
    torch.cuda.set_device(0)
    __graft_entry__.build()
    from paper_2008_12820_gb300 import claire, synth
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rows = []
    for n in (128, 256):
        w = synth.workload("blob256", shape=(n, n, n))
        shape = w["shape"]
        m0, m1 = torch.from_numpy(w["m0"]).cuda(), torch.from_numpy(w["m1"]).cuda()
        v = torch.zeros((3,) + shape, device="cuda")
        for beta in (5e-1, 1e-1, 5e-2):
            with claire.Registration(shape, w["nt"], beta, w["gamma"]) as reg:
                reg.set_images(m0, m1)
                for pc in ("invA", "invH0", "2LinvH0"):
                    v.zero_()
                    reg.solve(v, precond=pc)
                    torch.cuda.synchronize()
                    v.zero_()
                    e0.record(stream)
                    rep = reg.solve(v, precond=pc)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    rows.append({"n": n, "beta": beta, "precond": pc, "n_gn": rep.n_gn, "n_pcg": rep.n_pcg,
                                 "n_inner": rep.n_inner, "solve_ms": round(e0.elapsed_time(e1), 3),
                                 "t_pc_ms": round(rep.t_pc_ms, 3), "t_hess_ms": round(rep.t_hess_ms, 3),
                                 "grel": rep.grel, "status": rep.status})
    print(json.dumps({"study": "preconditioners (InvA, InvH0, 2LInvH0) on the synthetic blob pairs",
                      "nt": 4, "gamma": 1.0, "eps_n": 5e-2, "eps_h0": 1e-3, "rows": rows}), flush=True)


def run_precond(args):
    """(beta A)^-1 of a 3-component field alone (the five pencil passes of the
    inverse-A preconditioner, Section 3 "Preconditioning") on an n^3 grid
    (--grid, default 256), in a context with N_t = 1 so that little else is
    allocated: device time per application and the algorithmic bytes of the
    passes over it.  For profiling captures of the transform kernels at full
    size; not a bench line."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2008_12820_gb300 import claire
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    n = args.grid or 256
    shape = (n, n, n)
    rng = np.random.default_rng(5)
    r = torch.from_numpy(rng.standard_normal((3,) + shape).astype(np.float32)).cuda()
    s = torch.empty_like(r)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with claire.Registration(shape, 1, 1e-2, 1.0) as reg:
        for _ in range(args.warmup):
            reg.precond(r, out=s)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            reg.precond(r, out=s)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        h3 = n // 2 + 1
        # r2c: real in, half spectrum out; two c2c x2 passes and the x1 pass:
        # half spectrum in and out; c2r: half spectrum in, real out
        spec = 3 * n * n * h3 * 8
        real = 3 * n ** 3 * 4
        byts = (real + spec) + 2 * (2 * spec) + 2 * spec + (spec + real)
        print(json.dumps({"what": "(beta A)^-1 of a 3-component field, five pencil passes", "grid": list(shape),
                          "ms": round(ms, 4), "algorithmic_bytes": byts,
                          "workspace_gb": round(reg.workspace_bytes() / 1e9, 2),
                          "GBps": round(byts / (ms * 1e-3) / 1e9, 1)}), flush=True)


def run_oracle_study(args):
    """The FP64 oracle timed at the sizes the measurement plan names, on the
    host cores (OpenMP over all of them): gradient and one Hessian matvec at
    128^3 and 256^3 (v = half the generating velocity, a smooth direction),
    full solves from v = 0 at 32^3 and 128^3.  One JSON line; about half a
    minute of CPU work.  Context for the GPU numbers, not a bench line."""
    import numpy as np

    import oracle
    from paper_2008_12820_gb300 import synth
    oracle.build()
    rows = []
    for n in (128, 256):
        w = synth.workload(WORKLOAD, shape=(n, n, n))
        P = oracle.Problem(w["m0"], w["m1"], w["nt"], w["beta"], w["gamma"])
        v = (0.5 * w["v_true"]).astype(np.float64)
        vt = synth.smooth_direction((n, n, n), 7).astype(np.float64)
        t0 = time.perf_counter()
        P.gradient(v)
        t1 = time.perf_counter()
        P.matvec(vt)
        t2 = time.perf_counter()
        P.close()
        rows.append({"what": "gradient + matvec", "n": n, "gradient_s": round(t1 - t0, 3),
                     "matvec_s": round(t2 - t1, 3), "matvec_gvoxel_s": round(n ** 3 / (t2 - t1) / 1e9, 6)})
    for n in (32, 128):
        w = synth.workload("sin32" if n == 32 else WORKLOAD, shape=None if n == 32 else (n, n, n))
        P = oracle.Problem(w["m0"], w["m1"], w["nt"], w["beta"], w["gamma"])
        t0 = time.perf_counter()
        _, rep = P.solve(np.zeros((3,) + tuple(w["shape"])))
        t1 = time.perf_counter()
        P.close()
        rows.append({"what": "full solve from v = 0", "n": n, "workload": "sin32" if n == 32 else WORKLOAD,
                     "n_gn": rep.n_gn, "n_pcg": rep.n_pcg, "solve_s": round(t1 - t0, 3),
                     "gvoxel_s": round(n ** 3 / (t1 - t0) / 1e9, 7)})
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    print(json.dumps({"study": "FP64 oracle on the host cores", "cores": cores, "rows": rows}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch16":
        run_batch(args)
    elif args.workload == "pcstudy":
        run_pcstudy(args)
    elif args.workload == "oracle-study":
        run_oracle_study(args)
    elif args.workload == "precond":
        run_precond(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
