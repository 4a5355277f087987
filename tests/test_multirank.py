"""Host logic of the N > 1 benchmark path, run as two gloo ranks on the CPU.

The path does not shard: every rank detects its own frame on its own GPU
(independent replicas, no collective on the data path). What the ranks share
is the timing: a barrier around the timed region, the maximum of the ranks'
times, and the sum of the units they processed."""
import argparse
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    try:
        sys.path.insert(0, ROOT)
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                          WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
        import torch.distributed as dist

        import bench
        from paper_2307_16550_gb300 import scenes
        dist.init_process_group("gloo", rank=rank, world_size=world)
        w, r, _ = bench._dist()
        bench._barrier(w)
        # rank r "took" 10 * (r + 1) ms for 1000 * (r + 1) units
        value, ms_max, units = bench.aggregate(w, 10.0 * (r + 1), 1000 * (r + 1))
        sc = scenes.paper_frame(bench.replica_seed(r))
        q.put((r, value, ms_max, units, sc.targets.copy()))
        bench._barrier(w)
        dist.destroy_process_group()
    except Exception as e:  # reported to the parent
        q.put((rank, repr(e)))


def test_two_gloo_ranks_aggregate_as_replicas():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(2):
        item = q.get(timeout=120)
        assert len(item) == 5, f"rank {item[0]} failed: {item[1]}"
        out[item[0]] = item[1:]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        value, ms_max, units, _ = out[r]
        assert ms_max == 20.0  # the slowest rank's time
        assert units == 3000.0  # all ranks' units
        assert value == pytest.approx(3000.0 / 20e-3)
    # every rank detects its own frame
    assert not np.allclose(out[0][3], out[1][3])


def test_single_rank_aggregate_is_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(1, 4.0, 100) == (100 / 4e-3, 4.0, 100.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(gpus=2, steps=1, warmup=3, impl="reference", no_cpu_baseline=True)
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
