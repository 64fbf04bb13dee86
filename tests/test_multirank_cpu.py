"""The N > 1 path of bench.py on CPU: gloo ranks, each an independent
replica of the single domain (no data-path collective), the job time is the
slowest rank's, the batched workload's instances are split over the ranks
(each stepped exactly once, nodes balanced), and the reference arm runs on
rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, times, out):
    import torch.distributed as td
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_max = bench.max_over_ranks(times[rank], "cpu")
    value = bench.aggregate_mlups(1000, 10, ms_max, world)
    out.put((rank, ms_max, value))
    td.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_value():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [3.0, 5.0]
    ps = [ctx.Process(target=_worker, args=(r, world, port, times, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, value in res:
        assert ms_max == 5.0
        # 2 replicas x 1000 nodes x 10 steps in 5 ms
        assert value == pytest.approx(2 * 1000 * 10 / 5e-3 / 1e6)


def _shard_worker(rank, world, port, out):
    import torch
    import torch.distributed as td
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2005_08674_gb300 import inputs, lbm
    ws = inputs.batch_instances()
    cells = [w.nx * w.ny for w in ws]
    mine = bench.shard(cells, rank, world, lbm.lbm_partition_instances)
    # every rank "steps" its instances once: the sum over ranks must be one everywhere
    stepped = torch.zeros(len(ws), dtype=torch.int64)
    stepped[mine] += 1
    td.all_reduce(stepped)
    load = torch.tensor([float(sum(cells[k] for k in mine))], dtype=torch.float64)
    loads = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    td.all_gather(loads, load)
    out.put((rank, stepped.tolist(), [float(x) for x in loads], sum(cells)))
    td.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_batched_instances_shard_exactly_once_and_balance(world):
    """The batched mode's multi-rank split: each of the 256 instances is stepped
    by exactly one rank (no exchange needed: instances are independent), and the
    ranks' node counts agree within 5 % of the mean."""
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_shard_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = [q.get(timeout=180) for _ in range(world)]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, stepped, loads, total in res:
        assert stepped == [1] * len(stepped)
        assert sum(loads) == total
        mean = total / world
        assert max(abs(x - mean) for x in loads) <= 0.05 * mean, loads


def test_partition_rejects_bad_arguments():
    sys.path.insert(0, ROOT)
    from paper_2005_08674_gb300 import lbm
    assert lbm.lbm_partition_instances([], 4) == []
    assert lbm.lbm_partition_instances([5, 9, 1], 1) == [0, 0, 0]
    # largest first: 9 -> rank 0, 5 -> rank 1, 4 -> rank 1 (5 < 9), 1 -> rank 0 (9 = 9: lower rank)
    assert lbm.lbm_partition_instances([5, 9, 1, 4], 2) == [1, 0, 0, 1]
    for bad in ((([1, 2], 0)), (([1, -2], 2))):
        with pytest.raises(lbm.LbmError):
            lbm.lbm_partition_instances(*bad)


def test_reference_arm_rank_gating():
    """Under torchrun, rank 1 of the reference arm exits 0 without output."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_line():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "1"], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "MLUPS" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
