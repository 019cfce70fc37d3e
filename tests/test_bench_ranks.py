"""The multi-rank parts of bench.py on CPU: two gloo ranks agree on the
slowest rank's time, and the reference arm prints only on rank 0."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.sync_ranks(world, "cpu")
        mine = 10.0 + 7.5 * rank          # rank 1 is the slow one
        out[rank] = bench.max_over_ranks(mine, world, "cpu")
        bench.sync_ranks(world, "cpu")
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    world = 2
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world,
                       join=True, start_method="spawn")
    assert dict(out) == {0: 17.5, 1: 17.5}


def test_single_rank_helpers_need_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
    bench.sync_ranks(1, "cpu")


@pytest.mark.parametrize("rank,prints", [("1", False), ("0", True)])
def test_reference_arm_prints_on_rank_zero_only(rank, prints, tmp_path):
    env = dict(os.environ, RANK=rank, WORLD_SIZE="2", LOCAL_RANK=rank,
               DEC_INPUT_CACHE=str(tmp_path))
    args = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
            "--workload", "kuhn9", "--steps", "1", "--warmup", "0",
            "--ref-N", "5"]
    r = subprocess.run(args, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert (len(lines) == 1) == prints
    if prints:
        d = json.loads(lines[0])
        assert d["impl"] == "reference" and d["cpu_baseline"]["kind"] == "oracle"


def _shard_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ids = bench.rank_instances(3, rank, world)
        # stand-in for this rank's batched solve: k_eff of instance i
        k_local = [100.0 + i for i in ids]
        out[rank] = (ids, bench.gather_instances(k_local, world, "cpu").tolist())
    finally:
        dist.destroy_process_group()


def test_instances_split_across_two_gloo_ranks_and_gather_in_order():
    # 6 independent instances on 2 ranks: 3 + 3, k_eff gathered in global order
    world = 2
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_shard_main, args=(world, _free_port(), out), nprocs=world,
                       join=True, start_method="spawn")
    assert out[0][0] == [0, 1, 2] and out[1][0] == [3, 4, 5]
    assert out[0][1] == out[1][1] == [100.0, 101.0, 102.0, 103.0, 104.0, 105.0]
