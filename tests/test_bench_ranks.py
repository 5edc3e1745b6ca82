"""The multi-rank timing path of bench.py on CPU: two gloo ranks (one process
each, as torchrun starts them) reduce their timed-region lengths to the max
over ranks; the reported time per iteration is one replica's, and the
whole-job throughput counts every rank's replica."""
import multiprocessing as mp
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # rank r's timed region: 100 (r + 1) ms on the device, 150 + r ms of wall clock, 4 steps
        q.put((rank,) + bench.reduce_times(100.0 * (rank + 1), 150.0 + rank, 4, world, dist, "cpu"))
    finally:
        dist.destroy_process_group()


def test_reduce_times_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, dev, wall, per_step, iters_per_s, e2e in got:
        assert dev == 200.0 and wall == 151.0          # max over the ranks, the same on every rank
        assert per_step == 50.0                         # one replica's time per iteration
        assert iters_per_s == pytest.approx(40.0)       # 2 replicas x 4 iterations in 200 ms
        assert e2e == pytest.approx(151.0 / 4)          # one replica's wall time per iteration


def test_reduce_times_single_rank():
    import bench
    dev, wall, per_step, iters_per_s, e2e = bench.reduce_times(90.0, 120.0, 3, 1)
    assert (dev, wall, per_step, e2e) == (90.0, 120.0, 30.0, 40.0)
    assert iters_per_s == pytest.approx(3 / 0.09)


def test_reference_arm_line():
    """The reference arm (the oracle as it stands, on the host cores) prints
    one JSON line under the GPU arm's workload config, with a timed value,
    its sample and the e2e / cpu_baseline keys of the contract."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1",
                          "--ref-n", "10"], cwd=root, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads([ln for ln in out.stdout.splitlines() if ln.startswith("{")][-1])
    import bench
    assert line["impl"] == "reference"
    assert line["config"] == bench.workload_config(3, 32, 1)
    assert line["sample"]["n"] == 10 and line["value"] > 0 and line["ms_per_step"] == line["value"]
    assert line["higher_is_better"] is False and line["unit"] == "ms" and line["steps"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
