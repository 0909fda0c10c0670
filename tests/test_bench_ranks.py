"""The benchmark's multi-rank bookkeeping on CPU: two gloo ranks with different
step times agree on the slowest one, and the whole-job throughput counts every
rank's work (weak scaling, replicas of the same workload)."""
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


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.reduce_max(dist, 1.0 + rank, device="cpu")
    out[rank] = (t, bench.job_throughput(10 ** 9, world, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_step():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    assert out[0][0] == out[1][0] == 2.0
    assert out[0][1] == pytest.approx(world * 1.0 / 2.0)


def test_units_and_levels():
    import bench
    w = bench.WORKLOADS["headneck-256x256x128"]
    assert bench.schedule_units(w) == 956825600
    assert bench.level_dims((5, 3, 1), 3) == [(5, 3, 1), (3, 2, 1), (2, 1, 1)]


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the FP64 oracle on the host cores) prints one
    JSON line with the keys the benchmark contract names for the reference arm."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--workload", "headneck-256x256x128"], capture_output=True, text=True,
                         cwd=root, timeout=600, check=True)
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["host"]["nproc"] >= 1           # the host the oracle ran on
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] == "headneck-256x256x128"
    assert 1 <= d["cpu_baseline"]["cores"] <= d["cpu_baseline"]["host"]["nproc"]   # one process per core
    assert "processes" in d["cpu_baseline"]["sample"]


def test_default_workload_is_the_largest_single_gpu_configuration():
    import bench
    assert bench.DEFAULT_WORKLOAD == "large-512x512x256"
    sizes = {k: bench.schedule_units(w) for k, w in bench.WORKLOADS.items()}
    assert max(sizes, key=sizes.get) == bench.DEFAULT_WORKLOAD


def test_cpu_baseline_entry():
    """The bench's `cpu_baseline` entry (run after the GPU forms): the FP64 oracle
    on a bounded sample, with the host it ran on."""
    import bench
    w = bench.WORKLOADS["ellipsoid-64x64x32"]
    d = bench.cpu_baseline(w, bench.make_pair(w), budget_s=0.5)
    assert d["kind"] == "oracle" and d["cores"] >= 1 and d["value"] > 0
    assert d["unit"] == bench.UNIT and d["host"]["nproc"] >= 1 and "processes" in d["sample"]
    st = d["single_thread"]
    assert st["cores"] == 1 and st["value"] > 0 and "z-planes" in st["sample"]
