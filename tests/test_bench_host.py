"""Host logic of bench.py: throughput aggregation over ranks (gloo, world
size 2, on CPU), clock-record parsing and the roofline arithmetic."""

import os
import socket

import pytest

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r processed (r + 1) * 1000 vertex-frames in (r + 1) seconds
    v, t = bench.aggregate((rank + 1) * 1000.0, float(rank + 1), world, dist)
    q.put((rank, v, t))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for _, v, t in res:
        assert t == 2.0                     # max over ranks
        assert v == pytest.approx(3000.0 / 2.0)   # all vertex-frames / slowest time


def test_aggregate_single_rank():
    assert bench.aggregate(500.0, 2.0, 1) == (250.0, 2.0)


def test_parse_clock_rows():
    text = ("0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
            "0, 1980, 2070, 1300.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n"
            "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    r = bench.parse_clock_rows(text)
    assert r["sm_mhz"] == 2070 and r["sm_max_mhz"] == 2070 and r["samples"] == 3
    assert r["reasons"] == ["sw_power_cap"]


def test_roofline_arithmetic():
    prof = {"k_cg_L": (10, 2.0), "k_cg_LT": (10, 3.0), "k_cg_update": (10, 1.0),
            "k_cg_dir": (10, 0.5), "k_cg_alpha": (10, 0.1), "k_cg_beta": (10, 0.1)}
    stats = {"cg_iters_mean": 100.0, "cg_iters_max": 100}
    n, W, nnz, n_c = 1000000, 64, 6000000, 10
    r = bench.roofline(prof, stats, n, W, nnz, n_c, {"hbm_gbs": 6756.5}, single=False)
    assert r["kernel"] == "k_cg_LT" and r["bound"] == "alu"
    flops = n * W * (2 * 6 + 3) + n_c * W
    assert r["achieved"] == pytest.approx(flops / 0.3e-3 / 1e12, rel=1e-3)
    r = bench.roofline(prof, stats, n, W, nnz, n_c, {"hbm_gbs": 6756.5}, single=True)
    # FP32: the unweighted second pass reads degrees and anchor flags, no 1/d_i
    nbytes = n * W * 3 * 4 + 4 * (n + 1) + 4 * nnz + 5 * n
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(nbytes / 0.3e-3 / 1e9, rel=1e-3)
    assert abs(sum(r["time_share"].values()) - 1.0) < 1e-3


def test_stored_oracle_nmse_for_both_anchor_rules():
    for name in ("torus200x100_F256_k32", "grid316_F512_k64"):
        for key in (name, name + ":farthest"):
            sweeps, nmse = bench.nmse_reference(key)
            assert sweeps == bench.SWEEPS and 0.0 < nmse < 1.0
    assert bench.nmse_reference("no_such_workload") is None


@pytest.mark.parametrize("rule", ["random", "farthest"])
def test_oracle_leg_runs_with_either_anchor_rule(rule):
    smp = bench.sample_spec("icosphere4_F64_k16", 4, None, rule)
    res = bench.oracle_sample(smp, repeats=1)
    assert res["F"] == 4 and res["n"] == 2562 and len(res["times"]) == 1
    assert 0.0 <= res["nmse"] < 1.0


def test_oracle_leg_on_a_grid_patch():
    # the bounded sample of the large grid workloads: a corner patch with 1% anchors
    smp = bench.sample_spec("grid512_F300_k64", 3, 20, "random")
    res = bench.oracle_sample(smp, repeats=1)
    assert res["F"] == 3 and res["n"] == 400 and res["n_anchors"] == 4
    assert "20x20 corner patch" in bench.describe_sample(res, smp)


def test_roofline_scales_sampled_kernels_to_graph_iterations():
    # sampled kernels add up to 7.8 ms per iteration; the graph-replayed runs
    # took 3.9 ms per iteration: every kernel's time is halved, shares kept
    prof = {"k_cg_L": (10, 20.0), "k_cg_LT": (10, 30.0), "k_cg_update": (10, 20.0),
            "k_cg_dir": (10, 5.0), "k_cg_alpha": (10, 1.0), "k_cg_beta": (10, 2.0),
            "cg_iteration": (300, 1170.0)}
    stats = {"cg_iters_mean": 100.0, "cg_iters_max": 100}
    r = bench.roofline(prof, stats, 1000000, 64, 6000000, 10, {"hbm_gbs": 6756.5}, single=True)
    assert r["kernel"] == "k_cg_LT" and r["cg_iteration_ms"] == pytest.approx(3.9)
    assert r["mean_launch_ms"] == pytest.approx(1.5) and r["mean_launch_ms_event_bracketed"] == 3.0
    assert "cg_iteration" not in r["time_share"]


def test_workload_forms():
    # the default workload is the largest single-GPU one, in its benchmark form
    assert bench.DEFAULT_WORKLOAD == "grid512_F300_k64"
    f = bench.WORKLOAD_DEFAULTS[bench.DEFAULT_WORKLOAD]
    assert f["precision"] == "tf32" and f["refine"] > 0
    sweeps, nmse = bench.nmse_reference("grid512_F300_k64")
    assert sweeps == bench.SWEEPS and 0.0 < nmse < 1e-8
