"""The multi-rank path of bench.py on CPU: two gloo ranks, each a replica, time =
maximum over ranks, units = sum over ranks (the aggregation rank 0 reports)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, local = bench.dist_env()
    t, u = bench.reduce_max_sum(0.5 + rank, 1000 * (rank + 1))
    q.put((r, w, local, t, u))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_max_time_and_sum_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, world, local, t, u) in enumerate(out):
        assert rank == r and world == 2 and local == r
        assert t == pytest.approx(1.5) and u == pytest.approx(3000.0)


def test_reduce_is_identity_without_a_process_group():
    import bench
    assert bench.reduce_max_sum(0.25, 7) == (0.25, 7)


def test_bench_cli_and_legs_are_wired():
    import bench
    a = bench.parse_args(["--steps", "7", "--warmup", "3", "--leg", "adjoint", "--storage", "fp16",
                          "--grid", "32x8x8"])
    assert (a.steps, a.warmup, a.leg, a.storage, a.grid) == (7, 3, "adjoint", "fp16", "32x8x8")
    for name in ("forms_leg", "adjoint_leg", "large_leg", "moments_leg", "d2q33_leg", "e2e_leg", "cpu_baseline_leg",
                 "l2_assisted_leg", "run_reference", "run_ours"):
        assert callable(getattr(bench, name)), name
    assert len(bench.kernel_source_hash()) == 16


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` times the oracle on the host and prints one JSON line
    with the GPU arm's metric, unit and direction, an `impl` tag, a cpu_baseline that
    describes the run and an e2e entry without host-device traffic."""
    import json
    import os
    import subprocess
    import sys

    import bench
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                         cwd=root, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["unit"] == "MLUPS" and d["higher_is_better"] is True and d["n_gpus"] == 1
    assert (d["steps"], d["warmup"]) == (1, 0) and d["value"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # the reference arm prints our arm's config object for the same workload; the
    # sub-box it actually steps is named outside it
    from paper_1303_4624_gb300 import workloads as W
    assert d["config"]["workload"] == "d3q95_sweep_512x256x256"
    wl = W.Workload("d3q95_sweep_512x256x256", "D3Q95", "fp32", (512, 256, 256), 200, 1.8)
    assert d["config"] == bench.workload_config(wl, 95)
    assert d["sample_grid"].startswith("512x") and d["sample_grid"] in cb["sample"]
