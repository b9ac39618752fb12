"""Host logic of `bench.py --gpus N` ("replicas only": every rank advances its
own problem, no data exchange): the slowest rank's time is used and the
whole-job value counts every rank's zones.  Run as two gloo ranks on the CPU.
Also the reference arm under two ranks: rank 0 alone prints its line."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _max_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank            # rank 1 is the slowest
    got = bench.max_over_ranks_of(ms, dist, "cpu")
    value = bench.replica_throughput(world, 1000, 10, got)
    q.put((rank, got, value))
    dist.destroy_process_group()


def _reference_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank), OMP_NUM_THREADS="2")
    sys.path.insert(0, ROOT)
    import bench
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.main(["--impl", "reference", "--gpus", str(world), "--steps", "1", "--warmup", "1", "--n", "12"])
    q.put((rank, buf.getvalue()))


def _run(target, world=2):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    return [q.get(timeout=10) for _ in range(world)]


def test_slowest_rank_sets_the_time_and_value_counts_all_ranks():
    pytest.importorskip("torch")
    res = sorted(_run(_max_worker))
    for rank, got, value in res:
        assert got == 150.0
        assert value == pytest.approx(2 * 1000 * 10 / 0.150)


def test_reference_arm_prints_on_rank_zero_only():
    pytest.importorskip("torch")
    res = dict(_run(_reference_worker))
    assert res[1].strip() == ""
    line = json.loads(res[0].strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["unit"] == "zone-updates/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    # the oracle ran the workload the line names: its box, the steps it prints
    assert line["config"]["zones"] == 12 ** 3 and line["steps"] == 1 and line["warmup"] == 1
