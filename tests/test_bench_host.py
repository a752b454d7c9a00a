"""Host-side logic of bench.py without a GPU: the max-over-ranks timing
reduction of the multi-GPU (replica) path on two gloo ranks, the reference
arm's behaviour on ranks other than 0, the clock-sample parser, the per-
application projector accounting, the choice between the oracle's whole
reconstruction and its sample, and which workload the DRAM record and the
L2 note describe."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each rank reports its own p50, p99 and total; the job reports the slowest
        got = bench.max_over_ranks([10.0 + rank, 20.0 - rank, 3.0 * (rank + 1)], "cpu")
        out_q.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = dict(q.get(timeout=10) for _ in range(2))
    assert res[0] == res[1] == [11.0, 20.0, 6.0]


def test_max_over_ranks_without_process_group_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks([1.5, 2.0], "cpu") == [1.5, 2.0]


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=120, env=env)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_parse_clock_csv():
    sys.path.insert(0, ROOT)
    import bench

    text = "\n".join([
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ])
    c = bench.parse_clock_csv(text)
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"] and c["samples"] == 3
    assert bench.parse_clock_csv("") is None


def test_golden_nnz_count_is_the_oracles():
    """The roofline's algorithmic unit comes from tests/golden/nnz_counts.json;
    the 64^3 entry is recounted here with the oracle's walk."""
    import json
    import oracle as O
    import phantoms as P

    with open(os.path.join(ROOT, "tests", "golden", "nnz_counts.json")) as f:
        golden = json.load(f)
    scan = P.c1_small()
    rec = golden[scan.name]
    assert rec["M"] == scan.geometry.M and rec["N"] == scan.geometry.N
    assert O.count_nnz(scan.geometry) == rec["nnz"]
    for name, r in golden.items():  # every pieces count is at least one per hit ray and voxel
        assert r["nnz"] > max(r["M"], r["N"]) // 2, name


def test_code_digest_ignores_comments_only(tmp_path):
    sys.path.insert(0, ROOT)
    import bench

    a = tmp_path / "a.cu"
    a.write_text("// header\n__global__ void k(float *x) {\n    x[0] = 1.f;  // one\n}\n")
    b = tmp_path / "b.cu"
    b.write_text("/* other\n header */\n\n__global__ void k(float *x) {\n    x[0] = 1.f;\n}\n")
    c = tmp_path / "c.cu"
    c.write_text("__global__ void k(float *x) {\n    x[0] = 2.f;\n}\n")
    assert bench.code_digest(str(a)) == bench.code_digest(str(b))
    assert bench.code_digest(str(a)) != bench.code_digest(str(c))


def test_serving_patients_are_valid_and_seeded():
    sys.path.insert(0, ROOT)
    import bench
    import paper_2509_08574_gb300 as pk

    pats = bench.serving_patients()
    assert len(pats) == 16
    assert [p["geometry"].nx for p in pats] == [p["geometry"].nx for p in bench.serving_patients()]
    for p in pats:
        g = p["geometry"]
        assert g.nx in (128, 256, 384) and 30 <= g.n_views <= 120 and 256 <= g.nu <= 768
        assert 20 <= p["n_outer"] * p["n_inner"] <= 40
        pk.piccs_validate(g, pk.make_params(n_outer=p["n_outer"], n_inner=p["n_inner"]))


def test_projector_time_is_per_application_not_per_kernel():
    """One A^T is two kernels (ray scaling, gather) but one timed call: the
    per-application time must be the class total over its calls, so that
    time x applications gives back the class total."""
    sys.path.insert(0, ROOT)
    import bench

    # a 3 x 10 CGLS scan: 31 forward calls, 30 backprojections (60 kernels)
    prof = {"launches": {"forward": 31, "adjoint": 60},
            "calls": {"forward": 31, "adjoint": 30},
            "total_ms": {"forward": 31 * 5.36, "adjoint": 30 * 5.46}}
    per = bench.projector_ms_per_application(prof, 1)
    assert abs(per["forward"] - 5.36) < 1e-12
    assert abs(per["adjoint"] - 5.46) < 1e-12
    assert abs(per["adjoint"] * prof["calls"]["adjoint"] - prof["total_ms"]["adjoint"]) < 1e-9
    # a batched call serves B scans
    per4 = bench.projector_ms_per_application(prof, 4)
    assert abs(per4["adjoint"] - 5.46 / 4) < 1e-12


def test_both_arms_state_the_same_config():
    sys.path.insert(0, ROOT)
    import bench

    class A:
        workload, solver, batch, storage, seeds = "c2_needle", "cgls", 1, "f32", 10

    scan = bench.workload("c2_needle")
    cfg = bench.bench_config(scan, A)
    assert cfg == bench.bench_config(scan, A)
    assert cfg["noise_draws"] == 10 and cfg["batch"] == 1 and cfg["storage"] == "f32"
    assert "workspace" not in cfg["l2"]


def test_adjoint_kernel_label_follows_the_gather_choice():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.adjoint_kernel_names(bench.workload("c2_needle").geometry).startswith("scale_rays")
    assert bench.adjoint_kernel_names(bench.workload("c3_sphere_growth").geometry).startswith("scale_rays")
    assert bench.adjoint_kernel_names(bench.workload("c5_carm").geometry).startswith("ray_prefix")


def test_oracle_baseline_times_the_whole_reconstruction_when_it_is_short(monkeypatch):
    """The oracle's time per scan is its whole reconstruction where the
    sample estimates at most a minute for it, else the sample's estimate;
    the whole run gets the arm's solver."""
    sys.path.insert(0, ROOT)
    import bench

    calls = []
    monkeypatch.setattr(bench, "oracle_whole",
                        lambda scan, b, xp, solver=0: calls.append(solver) or (5.0, 1, "whole", 0.005))
    for est_ms, whole in ((1e3, True), (bench.ORACLE_WHOLE_MAX_S * 1e3, True), (5.6e5, False)):
        monkeypatch.setattr(bench, "oracle_sample", lambda scan, b, xp, e=est_ms: (e, 1, "sample", 1.0))
        calls.clear()
        got = bench.oracle_baseline(None, None, None, solver=2)
        assert (got[2] == "whole") == whole and calls == ([2] if whole else [])
        assert got[0] == (5.0 if whole else est_ms)


def test_metric_names_the_workload():
    sys.path.insert(0, ROOT)
    import bench

    class A:
        workload = "c2_needle"

    assert bench.metric_name(A, bench.workload("c2_needle")) == bench.METRIC
    A.workload = "c1_small"
    scan = bench.workload("c1_small")
    m = bench.metric_name(A, scan)
    assert m != bench.METRIC and scan.name in m and f"({scan.iterations} its)" in m


def test_traffic_record_is_the_workloads_own():
    """The committed DRAM counters describe one workload's launches: another
    workload (or a changed projector source) reports no traffic."""
    sys.path.insert(0, ROOT)
    import json

    import bench

    with open(os.path.join(ROOT, "profiles", "projector_traffic.json")) as f:
        rec = json.load(f)
    w = rec["bench_workload"]
    others = [k for k in bench.WORKLOADS if k != w]
    src = os.path.join(ROOT, "paper_2509_08574_gb300", "csrc", "kernels_project.cu")
    current = rec["code_sha256"] == bench.code_digest(src)
    for name in rec["kernels"]:
        assert (bench.traffic_record(name, w) is not None) == current
        for o in others:
            assert bench.traffic_record(name, o) is None


def test_l2_note_follows_the_working_set():
    sys.path.insert(0, ROOT)
    import bench

    assert "smaller than L2" in bench.l2_note(bench.workload("c1_small").geometry)
    assert "larger than L2" in bench.l2_note(bench.workload("c2_needle").geometry)
