"""The N > 1 bench path on CPU: two gloo ranks (127.0.0.1) each draw their own query
shard, and the whole-job time is the element-wise maximum over ranks (replicas with no
data-path collective; only the barrier and the max use the process group)."""
import importlib.util
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench = _bench()
        import synth
        assert bench.dist_setup() == (world, rank, rank)
        qs = bench.rank_query_sets(synth.small_grid(), 16, 3, rank, 0xB0)
        mine = torch.as_tensor(np.concatenate([np.stack([q.source, q.t_s]) for q in qs], axis=1)
                               .astype(np.int64))
        shards = [torch.zeros_like(mine) for _ in range(world)]
        dist.all_gather(shards, mine)
        times = bench.max_over_ranks([1.0 + rank, 10.0 - rank, 0.25 * (rank + 1)], world)
        dist.barrier()
        out.put((rank, [s.numpy() for s in shards], times))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_take_the_max():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    bench = _bench()
    import synth
    for rank, shards, times in res:
        assert times == [2.0, 10.0, 0.5]
        assert not np.array_equal(shards[0], shards[1])        # each rank its own queries
        for r in range(world):                                 # and the same as drawn alone
            alone = bench.rank_query_sets(synth.small_grid(), 16, 3, r, 0xB0)
            want = np.concatenate([np.stack([q.source, q.t_s]) for q in alone], axis=1)
            assert np.array_equal(shards[r], want)


def test_one_rank_needs_no_process_group():
    bench = _bench()
    assert bench.max_over_ranks([3.0, 4.0], 1) == [3.0, 4.0]
