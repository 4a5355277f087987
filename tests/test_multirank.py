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


# ---------------------------------------------------------------------------
# Sharded-grid argmax: one grid split over ranks, reduced by the packed key
# ---------------------------------------------------------------------------
def _split_grid_scores():
    """Hopping scores of a small frame from the oracle, with planted ties:
    the maximum repeated at a later cell of the other shard, and a tie of
    the second value straddling the shards."""
    sys.path.insert(0, ROOT)
    from oracle import hopping, maps, model
    from paper_2307_16550_gb300 import scenes
    radar = scenes.Radar(24e9, 250e6, 128e-6, 32, 16, 4)
    grid = scenes.Grid.from_bounds((0, 0, -10, -10), (20, 20, 10, 10), (6, 5, 4, 3))
    sc = scenes.custom_scene(7, radar, grid, Q=3, T=2, snr_db=10.0)
    Y = model.measurement(sc)
    S = hopping.hop_scores(maps.rd_maps(Y, 4), sc.radar, sc.tx, sc.rx, sc.grid).astype(np.float32).reshape(-1)
    return S


def _shard_main(rank, world, port, q, S, tie):
    try:
        sys.path.insert(0, ROOT)
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        import torch.distributed as dist

        from paper_2307_16550_gb300 import shard
        dist.init_process_group("gloo", rank=rank, world_size=world)
        S = S.copy()
        if tie:  # the maximum also at the last cell (shard 1) and at cell 1 (shard 0)
            S[-1] = S.max()
            S[1] = S.max()
        # rank r takes the (x, y) rows r, r + world, ... (every velocity cell of them)
        nv = 4 * 3
        cells = np.concatenate([np.arange(xy * nv, (xy + 1) * nv) for xy in range(rank, 30, world)])
        best = shard.local_argmax(S[cells], cells)
        q.put((rank, shard.allreduce_argmax(best), best))
        dist.destroy_process_group()
    except Exception as e:
        q.put((rank, repr(e), None))


@pytest.mark.parametrize("tie", [False, True])
def test_split_grid_argmax_by_packed_key(tie):
    import multiprocessing as mp
    S = _split_grid_scores()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_main, args=(r, 2, port, q, S, tie)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(2):
        r, glob, local = q.get(timeout=120)
        assert not isinstance(glob, str), f"rank {r} failed: {glob}"
        out[r] = (glob, local)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = S.copy()
    if tie:
        ref[-1] = ref.max()
        ref[1] = ref.max()
    want = (float(ref.max()), int(np.argmax(ref)))  # numpy: first index of the maximum
    assert out[0][0] == out[1][0] == want
    if tie:  # both shards hold the maximum (cell 1 on rank 0's rows, the last cell on rank 1's): cell 1 wins
        assert want[1] == 1
        assert out[0][1][0] == out[1][1][0] == want[0] and out[0][1][1] != out[1][1][1]


def test_packed_key_order():
    sys.path.insert(0, ROOT)
    from paper_2307_16550_gb300 import shard
    keys = [shard.pack_argmax_key(s, c) for s, c in [(0.0, 5), (0.0, 3), (1.5, 9), (1.5, 2), (2.0, 4000000000)]]
    # larger score first, then the smaller cell
    assert keys[1] > keys[0] and keys[2] > keys[1] and keys[3] > keys[2] and keys[4] > keys[3]
    for s, c in [(0.0, 0), (3.25, 17), (np.float32(1e30), 4294967294)]:
        assert shard.unpack_argmax_key(shard.pack_argmax_key(s, c)) == (float(np.float32(s)), c)
    assert shard.unpack_argmax_key(shard.NO_CANDIDATE) is None
    with pytest.raises(ValueError):
        shard.pack_argmax_key(-1.0, 0)
