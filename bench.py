#!/usr/bin/env python
"""Benchmark of the IRN-PICCS reconstruction path on GB300.

One step = one full IRN-PICCS reconstruction (3 reweighting cycles x 10 CGLS
iterations) of the 256^3 x 1 mm volume from 90 cone-beam views of 512 x 512
pixels (0.8 mm) over a 200 degree short scan, with every step of the path
(projector A, matched adjoint A^T, PICCS weights and stencils, Krylov vector
work) in this repository's CUDA kernels, inputs resident in HBM.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
instead: its whole reconstruction where that takes at most a minute (the 64^3
workload), else a bounded sample of the same workload.  Under torchrun every rank
runs an independent replica on its own GPU (the path has no exchange step).

Other measurements: `--solver lsqr|lsqr_reorth` (the inner solver),
`--storage bf16` (mixed precision, with its image error against FP32 and the
ground truth), `--batch B` (B scans per launch sequence), `--workload` (the
64^3, 512^3 and C-arm configurations), `--kernels-only` (the hot kernels
alone, for profiler captures) and `--serving` (a Poisson request stream over
16 patients through the request server against one scan at a time).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import re
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import phantoms as P  # noqa: E402

METRIC = "PICCS-Krylov recon ms/scan p50 at 256^3 (90 views of 512^2, 30 its)"
UNIT = "ms/scan"
L2_FLUSH_BYTES = 256 << 20
L2_BYTES = 129 * 10**6  # GB300's L2 (129 MB)
SOLVERS = {"cgls": (0, "CGLS"), "lsqr": (1, "LSQR"), "lsqr_reorth": (2, "re-orthogonalised LSQR")}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--seeds", type=int, default=10,
                    help="distinct noise draws of the scan the timed steps rotate through")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--solver", choices=list(SOLVERS), default="cgls",
                    help="inner Krylov solver (LSQR and CGLS are equivalent in exact arithmetic)")
    ap.add_argument("--workload", choices=list(WORKLOADS), default="c2_needle",
                    help="c2_needle: the 256^3 scan the headline is quoted on; c1_small: 64^3")
    ap.add_argument("--storage", choices=["f32", "bf16"], default="f32",
                    help="bf16: projections and the LSQR basis in BF16")
    ap.add_argument("--batch", type=int, default=1,
                    help="scans reconstructed together per step (one launch per kernel for all)")
    ap.add_argument("--serving", action="store_true",
                    help="request-stream benchmark: Poisson arrivals over 16 patients, served "
                         "(batching, overlap, graphs) against one scan at a time")
    ap.add_argument("--requests", type=int, default=64, help="--serving: requests in the stream")
    ap.add_argument("--rate", type=float, default=20.0, help="--serving: mean arrivals per second")
    ap.add_argument("--kernels-only", action="store_true",
                    help="run only the projector pair on the workload (for profiler captures)")
    return ap.parse_args()


WORKLOADS = {"c2_needle": P.c2_needle, "c1_small": P.c1_small,
             "c3_sphere_growth": P.c3_sphere_growth, "c5_carm": P.c5_carm}
# scans too large for the host's analytic line integrals: their data are made
# on the GPU (voxelised phantom, the projector, Poisson noise)
GPU_SYNTH = ("c3_sphere_growth", "c5_carm")


def workload(name="c2_needle"):
    return WORKLOADS[name]()


def workload_config(scan, solver="cgls"):
    g = scan.geometry
    return {
        "workload": (f"{scan.name}: {g.nx}^3 x {g.vx:g} mm volume, {g.n_views} views over "
                     f"{np.degrees((g.angles[1] - g.angles[0]) * g.n_views):.0f} deg, "
                     f"{g.nu}x{g.nv} detector x {g.du:g} mm, DSO {g.dso:g} / DSD {g.dsd:g} mm, "
                     f"IRN-PICCS {scan.n_outer} cycles x {scan.n_inner} "
                     f"{SOLVERS[solver][1]} iterations"),
        "solver": solver,
        "volume": [g.nx, g.ny, g.nz], "views": g.n_views, "detector": [g.nu, g.nv],
        "iterations": scan.iterations, "alpha": scan.alpha, "lambda": scan.lam, "tau": scan.tau,
        "projection_layout": "view,u,v (v fastest)",
        "l2": l2_note(g),
        "parallelism": "replicas (one independent reconstruction per GPU)",
    }


def l2_note(g):
    """How the L2 is kept from serving one step's inputs to the next: always
    a flush; whether the step's vectors alone (nine volume-sized and five
    projection-sized FP32 arrays) would exceed the L2 anyway is stated."""
    work = 4 * (9 * g.nx * g.ny * g.nz + 5 * g.n_views * g.nu * g.nv)
    note = f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write); "
    if work > L2_BYTES:
        return note + "working set larger than L2"
    return note + "working set smaller than L2 (the flush evicts it)"


def bench_config(scan, args):
    """The line's config, identical in both arms: the workload plus the run's
    batch, storage and number of noise draws."""
    draws = 1 if args.workload in GPU_SYNTH else max(1, args.seeds)
    return dict(workload_config(scan, args.solver), batch=max(1, args.batch),
                storage=args.storage, noise_draws=draws,
                value=("whole-job ms per scan: p50 step time (max over ranks) / "
                       "(ranks x scans per step); p50_ms/p99_ms: one replica's ms per scan"))


def nnz_of(scan):
    with open(os.path.join(ROOT, "tests", "golden", "nnz_counts.json")) as f:
        rec = json.load(f).get(scan.name)
    return int(rec["nnz"]) if rec else None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def code_digest(path):
    """sha256 of a C/CUDA source with its comments and blank lines removed, so
    that a comment edit does not invalidate counters taken on the same code."""
    with open(path) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    lines = [ln.rstrip() for ln in src.splitlines() if ln.strip()]
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()


def traffic_record(kernel, workload):
    """Per-launch DRAM traffic from a committed ncu summary, valid only for
    the workload it was taken on and while the projector code is unchanged
    since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "projector_traffic.json")
    src = os.path.join(ROOT, "paper_2509_08574_gb300", "csrc", "kernels_project.cu")
    try:
        with open(path) as f:
            rec = json.load(f)
        h = code_digest(src)
    except OSError:
        return None
    if rec.get("code_sha256") != h or rec.get("bench_workload") != workload:
        return None
    total = 0.0
    for name in kernel.split("+"):
        ent = rec.get("kernels", {}).get(name)
        if ent is None:
            return None
        total += float(ent["dram_bytes_per_launch"])
    return total


def parse_clock_csv(text):
    """Median SM clock, max clock and the throttle reasons seen, from the
    nvidia-smi CSV lines the sampler wrote (fields as ClockSampler.FIELDS)."""
    rows = []
    for line in text.splitlines():
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
        except ValueError:
            continue
    if not rows:
        return None
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for _, _, fl in rows for i, v in enumerate(fl)
                      if v.lower().startswith("active")})
    return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
            "reasons": reasons, "samples": len(rows)}


def max_over_ranks(values, device):
    """Element-wise maximum of a list of floats over all ranks (identity
    without an initialised process group); device is where the collective's
    tensor lives (cuda for NCCL, cpu for gloo)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.path = None
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
            sel = ["-i", uuid if uuid.startswith("GPU-") else "GPU-" + uuid]
        except Exception:
            sel = ["-i", str(device_index)]
        self.sel = sel

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", *self.sel, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        with open(self.path) as f:
            text = f.read()
        os.unlink(self.path)
        return parse_clock_csv(text)


def adjoint_kernel_names(g):
    """The two kernels of one backprojection on geometry g, by the library's
    choice: the prefix-sum gather for even nv and nz, at most one z crossing
    of a row per xy cell, nz <= 512 and at least 2.5 detector rows per voxel
    layer; the candidate gather otherwise."""
    vmax = 0.5 * (g.nv - 1) * g.dv
    multi = vmax > 0 and g.vz * g.dsd <= 1.01 * np.hypot(g.vx, g.vy) * vmax
    rows_per_layer = g.vz * g.dsd / (g.dso * g.dv)
    if g.nv % 2 == 0 and g.nz % 2 == 0 and not multi and g.nz <= 512 and rows_per_layer >= 2.5:
        return "ray_prefix_kernel+adj_prefix_kernel"
    return "scale_rays_kernel+adj_gather_kernel"


def projector_ms_per_application(prof, batch):
    """Device ms of one application of A and of A^T per scan, from a library
    profile: each class's summed time over its operator calls (not its kernel
    launches -- one A^T is two kernels), divided by the scans one batched call
    serves."""
    per = {}
    for kind in ("forward", "adjoint"):
        n = prof["calls"][kind]
        per[kind] = (prof["total_ms"][kind] / n / batch) if n else float("nan")
    return per


def pctl(xs, q):
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q))


# --------------------------------------------------------------------------
# CPU oracle sample (cpu_baseline and the reference arm)
# --------------------------------------------------------------------------
def metric_name(args, scan):
    """The headline metric on the 256^3 workload, else the workload's own."""
    if args.workload == "c2_needle":
        return METRIC
    return f"PICCS-Krylov recon ms/scan p50, {scan.name} ({scan.iterations} its)"


def oracle_sample(scan, b, xp):
    """Times the FP64 oracle on a bounded sample of the workload: A and A^T on
    one view in ten, plus one pass of the regularisation blocks over the full
    volume; extrapolated to a whole reconstruction."""
    import oracle as O

    g = scan.geometry
    sub = list(range(0, g.n_views, 10))
    gs = g.replace(angles=g.angles[sub])
    bsub = np.ascontiguousarray(b[sub], dtype=np.float64)
    x64 = xp.astype(np.float64)
    t0 = time.perf_counter()
    O.forward(gs, x64)
    t1 = time.perf_counter()
    O.adjoint(gs, bsub)
    t2 = time.perf_counter()
    g3 = O.grad(x64)
    w = O.weights(g3, scan.tau)
    O.grad_adj(w[None] * g3)
    O.grad_adj(w[None] * g3)
    t3 = time.perf_counter()
    scale = g.n_views / len(sub)
    pair = scale * ((t1 - t0) + (t2 - t1)) + (t3 - t2)
    # explicit-residual CGLS: one (A, A^T) pair to restart each cycle plus one
    # per iteration
    per_scan_s = scan.n_outer * (scan.n_inner + 1) * pair
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = (f"A and A^T on {len(sub)} of {g.n_views} views plus one regularisation pass on the "
              f"full {g.nx}^3 volume ({t3 - t0:.1f} s), scaled to {scan.n_outer}x"
              f"({scan.n_inner}+1) projector pairs per scan")
    return per_scan_s * 1e3, cores, sample, t3 - t0


# a whole oracle reconstruction is timed instead of the sample when the
# sample's estimate of it is at most this long
ORACLE_WHOLE_MAX_S = 60.0


def oracle_whole(scan, b, xp, solver=0):
    """Times the FP64 oracle's whole reconstruction of the workload: the same
    projections, prior, parameters and solver as the GPU arm, end to end."""
    import oracle as O

    g = scan.geometry
    x64 = xp.astype(np.float64)
    t0 = time.perf_counter()
    O.irn(g, np.ascontiguousarray(b, dtype=np.float64), x64, x64, scan.alpha, scan.lam, scan.tau,
          scan.n_outer, scan.n_inner, solver=solver)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    name = next(v[1] for v in SOLVERS.values() if v[0] == solver)
    sample = (f"the whole reconstruction, {scan.n_outer}x{scan.n_inner} {name} iterations on the "
              f"{g.nx}x{g.ny}x{g.nz} workload ({dt:.1f} s)")
    return dt * 1e3, cores, sample, dt


def oracle_baseline(scan, b, xp, solver=0):
    """The oracle's time per scan: its whole reconstruction when the sample
    estimates that at ORACLE_WHOLE_MAX_S or less, else the sample's estimate."""
    est = oracle_sample(scan, b, xp)
    if est[0] <= ORACLE_WHOLE_MAX_S * 1e3:
        return oracle_whole(scan, b, xp, solver)
    return est


def oracle_sample_1thread(scan, b, xp):
    """The oracle's projector pair on one thread, on one view: ms per scan
    extrapolated like oracle_sample (the regularisation pass is left out; it is
    under 1 % of the oracle's time)."""
    import oracle as O

    g = scan.geometry
    gs = g.replace(angles=g.angles[:1])
    x64 = xp.astype(np.float64)
    t0 = time.perf_counter()
    O.forward(gs, x64, nthreads=1)
    O.adjoint(gs, np.ascontiguousarray(b[:1], dtype=np.float64), nthreads=1)
    dt = time.perf_counter() - t0
    return scan.n_outer * (scan.n_inner + 1) * g.n_views * dt * 1e3, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    scan = workload(args.workload)
    b = scan.measured()
    xp = scan.prior_volume(ss=1)
    solver = SOLVERS[args.solver][0]
    for _ in range(args.warmup):
        oracle_baseline(scan, b, xp, solver)
    vals = []
    cores = sample = None
    for _ in range(args.steps):
        v, cores, sample, _ = oracle_baseline(scan, b, xp, solver)
        vals.append(v)
    value = pctl(vals, 50)
    line = {
        "impl": "reference", "metric": metric_name(args, scan), "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": value, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(scan, args),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# our CUDA path
# --------------------------------------------------------------------------
def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_2509_08574_gb300 as pk

    scan = workload(args.workload)
    g = scan.geometry
    t_in = time.perf_counter()
    truth = None
    if args.workload in GPU_SYNTH:
        b, xp, truth = synth_inputs(scan, pk, torch)
        b_np = xp_np = None
    else:
        # the analytic line integrals once, then one Poisson draw per seed
        li = P.project_analytic(scan.scan_phantom, g)
        draws = [P.poisson_log_data(li, scan.I0, scan.noise_seed + k).astype(np.float32)
                 for k in range(max(1, args.seeds))]
        b_np = draws[0]
        xp_np = scan.prior_volume(ss=1)  # the oracle's timing sample reads this one
        b = torch.from_numpy(b_np).cuda()
        if scan.prior_file is None and args.workload in DENSE_PRIOR_VIEWS:
            xp = dense_scan_prior(scan, DENSE_PRIOR_VIEWS[args.workload], pk, torch)
        else:
            xp = torch.from_numpy(xp_np).cuda()
    t_in = time.perf_counter() - t_in

    stream = torch.cuda.Stream()
    B = max(1, args.batch)
    if B > 1:  # B scans of the workload, reconstructed together
        b = b.unsqueeze(0).expand((B,) + tuple(b.shape)).contiguous()
        xp = xp.unsqueeze(0).expand((B,) + tuple(xp.shape)).contiguous()
    out = torch.empty(((B,) if B > 1 else ()) + g.vol_shape(), dtype=torch.float32, device="cuda")
    # the timed steps rotate through the noise draws (one scan's worth each)
    inputs = [b]
    if b_np is not None and args.seeds > 1:
        for d in draws[1:]:
            t = torch.from_numpy(d).cuda()
            inputs.append(t.unsqueeze(0).expand((B,) + tuple(t.shape)).contiguous() if B > 1 else t)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    storage = pk.STORAGE_BF16 if args.storage == "bf16" else pk.STORAGE_F32
    params = pk.make_params(scan.alpha, scan.lam, scan.tau, scan.n_outer, scan.n_inner,
                            solver=SOLVERS[args.solver][0], storage=storage)
    torch.cuda.synchronize()
    ctx = pk.Context(g, stream=stream, batch=B)
    ctx.set_prior(xp)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.zero_()
            ctx.reconstruct(b, params, out=out)
    stream.synchronize()
    for slot in range(B):
        rep = ctx.report(slot)
        if rep.status != 0 or rep.iterations_run != scan.iterations:
            raise RuntimeError(f"reconstruction {slot}: status {rep.status}, "
                               f"{rep.iterations_run} iterations")
    with torch.cuda.stream(stream):  # every noise draw reconstructs cleanly too
        for inp in inputs[1:]:
            ctx.reconstruct(inp, params, out=out)
            if ctx.report().status != 0:
                raise RuntimeError("reconstruction of a noise draw failed")

    clocks = ClockSampler(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    ctx.profile_enable(True)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.zero_()  # outside the step's events: L2 holds no input at step start
            ev[k][0].record(stream)
            ctx.reconstruct(inputs[k % len(inputs)], params, out=out)
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    prof = ctx.profile_read()
    step_ms = [a.elapsed_time(c) / B for a, c in ev]  # per scan
    p50, p99 = pctl(step_ms, 50), pctl(step_ms, 99)
    total_ms = float(sum(step_ms))

    p50, p99, total_ms = max_over_ranks([p50, p99, total_ms], "cuda")

    # end to end through the public API with host buffers (copies inside)
    if args.e2e_steps > 0:
        hb = b.cpu().pin_memory()
        hout = torch.empty(tuple(out.shape), dtype=torch.float32).pin_memory()
    ctx.set_stream(stream)
    e2e_ms = []
    for k in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        with torch.cuda.stream(stream):
            flush.zero_()
        stream.synchronize()
        t0 = time.perf_counter()
        ctx.reconstruct_host(hb, params, out=hout)
        dt = (time.perf_counter() - t0) * 1e3 / B
        if k > 0:  # first call warms the pinned-memory path
            e2e_ms.append(dt)
    e2e_p50 = max_over_ranks([pctl(e2e_ms, 50)], "cuda")[0] if e2e_ms else None

    # roofline of the dominant kernel (measured live inside the timed region)
    nnz = nnz_of(scan)
    peaks, peak_kind = measured_peaks()
    per = projector_ms_per_application(prof, B)
    dom = max(("forward", "adjoint"), key=lambda k: prof["total_ms"][k])
    nz_ = nnz if nnz is not None else float("nan")  # no exact count: no roofline
    alg_bytes = 4.0 * (nz_ + g.M + g.N)
    achieved = alg_bytes / (per[dom] * 1e-3) / 1e9
    peak = float(peaks["hbm_gbs"])
    kernel_names = {"forward": "fwd_kernel", "adjoint": adjoint_kernel_names(g)}

    line = {
        "metric": metric_name(args, scan),
        # whole job: every rank reconstructs B scans per step, so the job's time
        # per scan is the (slowest rank's) step time over all ranks' scans
        "value": p50 / world, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms * B / args.steps, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": bench_config(scan, args),
        "workspace_bytes": int(pk.piccs_query_workspace_batched(g, params, B)),
        "p50_ms": p50, "p99_ms": p99,
        "job_scans_per_s": world * args.steps * B / (total_ms * B * 1e-3),
        "e2e": {"value": e2e_p50, "unit": UNIT, "h2d_bytes_per_step": int(B * g.N * 4),
                "d2h_bytes_per_step": int(B * g.M * 4)} if e2e_p50 is not None else None,
        "gpu_launches": int(prof["total_launches"]),
        "kernel_ms_per_step": {k: v / args.steps for k, v in prof["total_ms"].items()},
        "kernel_ms_per_scan": {k: v / args.steps / B for k, v in prof["total_ms"].items()},
        "launches_per_step": {k: v / args.steps for k, v in prof["launches"].items()},
        "calls_per_step": {k: v / args.steps for k, v in prof["calls"].items()},
        "projector": {"nnz": nnz, "fwd_ms": per["forward"], "adj_ms": per["adjoint"],
                      "fwd_gups": nz_ / (per["forward"] * 1e-3) / 1e9,
                      "adj_gups": nz_ / (per["adjoint"] * 1e-3) / 1e9},
        "roofline": {"kernel": kernel_names[dom], "bound": "hbm", "achieved": achieved,
                     "peak": peak, "peak_source": f"{peak_kind} hbm_gbs", "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic_record(kernel_names[dom], args.workload),
                     "algorithmic_bytes_per_launch": alg_bytes},
        "clocks": clk,
        "wall_s_timed_region": t_wall, "input_generation_s": t_in,
    }
    if storage == pk.STORAGE_BF16 and rank == 0:
        # image error of the BF16 path: against the FP32 path and the ground truth
        with torch.cuda.stream(stream):
            xb = ctx.reconstruct(b, params, out=out).clone()
            p32 = pk.make_params(scan.alpha, scan.lam, scan.tau, scan.n_outer, scan.n_inner,
                                 solver=SOLVERS[args.solver][0])
            x32 = ctx.reconstruct(b, p32, out=out).clone()
        stream.synchronize()
        xb, x32 = xb.reshape(-1, g.M)[0].double(), x32.reshape(-1, g.M)[0].double()
        truth = (truth.reshape(-1).double() if truth is not None else
                 torch.from_numpy(scan.truth_volume(ss=1).reshape(-1)).double().cuda())
        rel = lambda a, c: float(torch.linalg.norm(a - c) / torch.linalg.norm(c))
        line["error"] = {"rel_l2_bf16_vs_f32": rel(xb, x32),
                         "rel_l2_to_truth": {"f32": rel(x32, truth), "bf16": rel(xb, truth)}}
        line["dtype"] = "bf16 storage, f32 accumulation, f64 scalars"
    if scan.prior_file is not None:
        line["prior"] = "stored fixture: reconstructed by the oracle from a dense scan"
    elif args.workload in DENSE_PRIOR_VIEWS:
        line["prior"] = (f"reconstructed on the GPU from {DENSE_PRIOR_VIEWS[args.workload]} views over "
                         "360 deg of the change-free phantom (20 plain CGLS iterations)")
    else:
        line["prior"] = "change-free phantom voxelised at voxel centres"
    if args.workload in GPU_SYNTH:
        line["data"] = "synthetic (phantom voxelised on the GPU, projected by this projector, Poisson noise)"
    if rank == 0 and world == 1 and not args.no_cpu_baseline and b_np is not None:
        v, cores, sample, _ = oracle_baseline(scan, b_np, xp_np, SOLVERS[args.solver][0])
        v1, dt1 = oracle_sample_1thread(scan, b_np, xp_np)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": sample,
                                "one_thread": {"value": v1, "unit": UNIT, "cores": 1,
                                               "sample": f"A and A^T on 1 of {scan.geometry.n_views} "
                                                         f"views on one thread ({dt1:.1f} s)"}}
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_kernels_only(args):
    """The hot kernels alone on the workload, each launch preceded by an L2
    flush: A (forward), A^T (adjoint), the regularisation normal operator
    D^T Omega D z with its energy (reg_normal) and the IRN reweighting
    (weights + prior right-hand side); prints their CUDA-event times."""
    import torch
    import paper_2509_08574_gb300 as pk

    scan = workload(args.workload)
    g = scan.geometry
    x = torch.from_numpy(scan.prior_volume(ss=1)).cuda()
    y = torch.from_numpy(P.random_projections(g, 7).astype(np.float32)).cuda()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    q = torch.empty(g.proj_shape(), dtype=torch.float32, device="cuda")
    s = torch.empty(g.vol_shape(), dtype=torch.float32, device="cuda")
    params = pk.make_params(scan.alpha, scan.lam, scan.tau, 1, 1)
    stream = torch.cuda.current_stream()
    with pk.Context(g, stream=stream) as ctx:
        ctx.set_prior(x)
        z = 1.01 * x
        omega, c = ctx.reg_weights(z, params)
        t = torch.empty_like(z)
        times = {"forward": [], "adjoint": [], "reg_normal": [], "reweight": []}
        for _ in range(max(args.steps, 1)):
            for kind in times:
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                if kind == "forward":
                    ctx.forward(x, q)
                elif kind == "adjoint":
                    ctx.adjoint(y, s)
                elif kind == "reg_normal":
                    pk.piccs_reg_normal(ctx.h, omega, params, z, t, False)
                else:
                    ctx.reg_weights(z, params, omega, c)
                e1.record()
                torch.cuda.synchronize()
                times[kind].append(e0.elapsed_time(e1))
    print(json.dumps({k: {"ms": v} for k, v in times.items()}), flush=True)
    return 0


# --------------------------------------------------------------------------
# request stream (serving)
# --------------------------------------------------------------------------
def serving_patients(n_patients=16, seed=4):
    """Seeded patient mix: volumes 128^3 / 256^3 / 384^3 (1 mm), 30-120 views
    (200 or 360 deg), square detectors 256-768 pixels sized to cover the
    volume, 20-40 iterations (2-4 cycles of 10)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pats = []
    for k in range(n_patients):
        n = int(rng.choice([128, 256, 384]))
        views = int(rng.integers(30, 121))
        det = int(rng.choice([256, 384, 512, 640, 768]))
        arc = float(rng.choice([200.0, 360.0]))
        du = 1.1 * n * 1.0 * 1.5 / det  # magnification 1.5, 10 % margin
        g = P.Geometry(n, n, n, 1.0, 1.0, 1.0, det, det, du, du, 1000.0, 1500.0,
                       P.scan_angles(views, arc))
        pats.append(dict(geometry=g, n_outer=int(rng.integers(2, 5)), n_inner=10, seed=100 + k))
    return pats


def _voxelize_gpu(phantom, g, torch):
    """Ellipsoid / cylinder phantom sampled at voxel centres on the GPU (input
    synthesis), z slab by z slab."""
    vol = torch.zeros((g.nx, g.ny, g.nz), dtype=torch.float32, device="cuda")
    ax = [((torch.arange(n, device="cuda", dtype=torch.float32) + 0.5) - n / 2.0) * v
          for n, v in ((g.nx, g.vx), (g.ny, g.vy), (g.nz, g.vz))]
    for z0 in range(0, g.nz, 64):
        X, Y, Z = torch.meshgrid(ax[0], ax[1], ax[2][z0:z0 + 64], indexing="ij")
        for e in phantom:
            if isinstance(e, P.Cylinder):
                a = torch.tensor(e.p1 - e.p0, dtype=torch.float32, device="cuda")
                h = float(torch.linalg.norm(a))
                a = a / h
                rx, ry, rz = X - float(e.p0[0]), Y - float(e.p0[1]), Z - float(e.p0[2])
                ra = rx * a[0] + ry * a[1] + rz * a[2]
                rp2 = rx * rx + ry * ry + rz * rz - ra * ra
                ins = (ra >= 0) & (ra <= h) & (rp2 <= e.radius ** 2)
            else:
                c = [float(t) for t in e.center]
                R = torch.tensor(e.rot, dtype=torch.float32, device="cuda")
                q = torch.zeros_like(X)
                for k in range(3):
                    qk = ((X - c[0]) * R[0, k] + (Y - c[1]) * R[1, k] + (Z - c[2]) * R[2, k]) / float(e.semi[k])
                    q += qk * qk
                ins = q <= 1.0
            vol[:, :, z0:z0 + 64] += float(e.mu) * ins.float()
    return vol


# workloads whose prior is reconstructed from a dense scan of the change-free
# phantom at run time (the 64^3 workload stores its prior, made by the oracle)
DENSE_PRIOR_VIEWS = {"c2_needle": 720}


def dense_scan_prior(scan, views, pk, torch, iters=20):
    """The workload's prior: the change-free phantom scanned with `views`
    views over 360 degrees on the same detector (voxelised on the GPU,
    projected by this library's A, Poisson noise at the workload's I0) and
    reconstructed by `iters` plain CGLS iterations (alpha = lambda = 0) from
    zero, on the GPU."""
    g = scan.geometry.replace(angles=P.scan_angles(views, 360.0))
    ph = _voxelize_gpu(scan.prior_phantom, g, torch)
    with pk.Context(g) as ctx:
        li = ctx.forward(ph)
        gen = torch.Generator(device="cuda").manual_seed(scan.noise_seed + 1000)
        b = -torch.log(torch.clamp(torch.poisson(scan.I0 * torch.exp(-li), generator=gen), min=1.0)
                       / scan.I0)
        del li
        ctx.set_prior(torch.zeros_like(ph))
        x = ctx.reconstruct(b, pk.make_params(0.0, 0.0, scan.tau, 1, iters,
                                              x0_mode=pk.X0_ZERO, variant=pk.VARIANT_CGLS))
        if ctx.report().status != 0:
            raise RuntimeError("dense-scan prior reconstruction failed")
    torch.cuda.synchronize()
    return x


def synth_inputs(scan, pk, torch):
    """(b, x_p, x_true) on the GPU: the change-free and the changed phantoms
    voxelised at voxel centres, b = -log(Poisson(I0 exp(-A x_true)) / I0)."""
    g = scan.geometry
    xp = _voxelize_gpu(scan.prior_phantom, g, torch)
    xt = _voxelize_gpu(scan.scan_phantom, g, torch)
    with pk.Context(g) as ctx:
        li = ctx.forward(xt)
    gen = torch.Generator(device="cuda").manual_seed(scan.noise_seed)
    b = -torch.log(torch.clamp(torch.poisson(scan.I0 * torch.exp(-li), generator=gen), min=1.0)
                   / scan.I0)
    del li
    return b, xp, xt


def run_serving(args):
    import threading
    import torch
    import paper_2509_08574_gb300 as pk

    pats = serving_patients()
    t_in = time.perf_counter()
    data = []
    for p in pats:
        g = p["geometry"]
        prior_ph = P.ellipsoid_phantom(g, 12, seed=p["seed"], body_mu=0.02)
        change = P.Ellipsoid(np.array([0.1, -0.05, 0.0]) * g.nx, np.array([4.0, 4.0, 4.0]),
                             np.eye(3), 0.01)
        xp = _voxelize_gpu(prior_ph, g, torch)
        xt = xp + _voxelize_gpu([change], g, torch)
        with pk.Context(g) as ctx:
            li = ctx.forward(xt)
        gen = torch.Generator(device="cuda").manual_seed(p["seed"])
        counts = torch.poisson(5e4 * torch.exp(-li), generator=gen)
        b = -torch.log(torch.clamp(counts, min=1.0) / 5e4)
        data.append(dict(prior=xp.cpu().numpy(), proj=b.cpu().pin_memory(),
                         proj16=b.to(torch.bfloat16).cpu().pin_memory(),
                         params=pk.make_params(0.5, 0.5, 1e-2, p["n_outer"], p["n_inner"],
                                               solver=SOLVERS[args.solver][0])))
        del xp, xt, li, counts, b
    torch.cuda.synchronize()
    t_in = time.perf_counter() - t_in
    rng = np.random.Generator(np.random.PCG64(9))
    arrivals = np.cumsum(rng.exponential(1.0 / args.rate, size=args.requests))
    who = rng.integers(0, len(pats), size=args.requests)

    def outbufs():
        return [[torch.empty(p["geometry"].vol_shape(), dtype=torch.float32).pin_memory()
                 for _ in range(2)] for p in pats]

    clocks = ClockSampler(0)  # over every arm
    clocks.start()
    # plain: one scan at a time in arrival order, sessions resident, no batching
    outs = outbufs()
    ctxs = []
    for p, d in zip(pats, data):
        c = pk.Context(p["geometry"])
        c.set_prior(torch.from_numpy(d["prior"]).cuda())
        ctxs.append(c)
    for k in range(len(pats)):  # warm the path once per patient
        ctxs[k].reconstruct_host(data[k]["proj"], data[k]["params"], out=outs[k][0])
    lat_plain = []
    t0 = time.perf_counter()
    for r in range(args.requests):
        now = time.perf_counter() - t0
        if now < arrivals[r]:
            time.sleep(arrivals[r] - now)
        k = int(who[r])
        ctxs[k].reconstruct_host(data[k]["proj"], data[k]["params"], out=outs[k][r % 2])
        lat_plain.append((time.perf_counter() - t0 - arrivals[r]) * 1e3)
    span_plain = time.perf_counter() - t0
    for c in ctxs:
        c.close()
    torch.cuda.synchronize()

    def summary(lat, span):
        return {"p50_ms": pctl(lat, 50), "p99_ms": pctl(lat, 99),
                "scans_per_s": args.requests / span, "makespan_s": span}

    # served: the request loop (FP32 storage, then BF16 storage with BF16 inputs)
    def served_arm(bf16, order=pk.ORDER_ADAPTIVE, max_group=1):
        outs = outbufs()
        srv = pk.Server(max_batch=8, max_running=2, use_graphs=True, order=order,
                        max_group=max_group)
        prm = []
        for k, (p, d) in enumerate(zip(pats, data)):
            srv.add_patient(k, p["geometry"], d["prior"])
            q = d["params"]
            prm.append(pk.make_params(q.alpha, q.lambda_, q.tau, q.n_outer, q.n_inner,
                                      solver=q.solver,
                                      storage=pk.STORAGE_BF16 if bf16 else pk.STORAGE_F32))
        src = "proj16" if bf16 else "proj"
        for k in range(len(pats)):  # warm: sessions resident, graphs captured for batch 1
            t, _ = srv.submit(k, data[k][src], prm[k], out=outs[k][0])
            srv.wait(t)
        warm = srv.stats()
        tickets = [None] * args.requests
        t0 = time.perf_counter()

        def feeder():
            for r in range(args.requests):
                now = time.perf_counter() - t0
                if now < arrivals[r]:
                    time.sleep(arrivals[r] - now)
                k = int(who[r])
                tickets[r] = srv.submit(k, data[k][src], prm[k], out=outs[k][r % 2])[0]

        th = threading.Thread(target=feeder)
        th.start()
        th.join()
        st = [srv.wait(t) for t in tickets]
        span = time.perf_counter() - t0
        sstats = srv.stats()
        srv.close()
        if any(x["status"] != 0 for x in st):
            raise RuntimeError("served request failed")
        res = summary([x["total_ms"] for x in st], span)
        res.update(max_batch=8, max_running=2, max_group=max_group, graphs=True,
                   storage="bf16" if bf16 else "f32",
                   order={pk.ORDER_FIFO: "fifo", pk.ORDER_RESPONSE_RATIO: "response_ratio"}.get(
                       order, "adaptive"),
                   mean_batch=args.requests / max(sstats["batches"] - warm["batches"], 1),
                   server=sstats)
        return res

    served, served16 = served_arm(False), served_arm(True)
    served_rr = served_arm(False, pk.ORDER_RESPONSE_RATIO)
    served_grp = served_arm(False, max_group=4)
    clk = clocks.stop()
    plain = summary(lat_plain, span_plain)
    line = {
        "metric": "serving latency p50/p99 and scans/s (Poisson request stream, 16 patients)",
        "value": served["p50_ms"], "unit": "ms", "higher_is_better": False, "n_gpus": 1,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{args.requests} requests, Poisson arrivals {args.rate:g}/s over "
                               f"{len(pats)} patients: 128^3/256^3/384^3 x 1 mm volumes, 30-120 "
                               "views, 256^2-768^2 detectors, 20-40 iterations",
                   "solver": args.solver,
                   "patients": [[p["geometry"].nx, p["geometry"].n_views, p["geometry"].nu,
                                 p["n_outer"] * p["n_inner"]] for p in pats]},
        "served": served,
        "served_bf16": served16,
        "served_response_ratio": served_rr,
        "served_grouped": served_grp,
        "plain_one_at_a_time": plain,
        "clocks": clk,
        "input_generation_s": t_in,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse_args()
    if args.kernels_only:
        return run_kernels_only(args)
    if args.serving:
        return run_serving(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
