"""Multi-rank replica logic of the benchmark on CPU (gloo, world size 2).

Colourings are independent (Algorithm 1's outer loop), so N GPUs run N
replicas on disjoint colouring ranges and the job time is the max over ranks;
there is no collective on the data path.  This checks the sharding, the
max-reduction and the cross-check of per-colouring results gathered on rank 0
(which recounts one colouring of every other rank) with two real processes."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, steps, n_iter, q, bad):
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ranges = [(bench.replica_first_iter(rank, world, i, n_iter), n_iter) for i in range(steps)]
    everything = [None] * world
    dist.all_gather_object(everything, ranges)
    tmax = bench.max_over_ranks(1.5 + rank)
    # per-colouring results of each rank, gathered on rank 0 and cross-checked
    # by recounting: a stand-in count that depends on the colouring index only,
    # and a rank 1 that planted a wrong count
    def count(j):
        return (j * 2654435761) % 1000003

    mine = [(j, count(j) + (1 if (rank == 1 and bad) else 0)) for a, n in ranges for j in range(a, a + n)]
    per_rank = [None] * world
    dist.all_gather_object(per_rank, mine)
    if rank == 0:
        q.put((everything, tmax, bench.replica_check(per_rank, count)))
    dist.barrier()
    dist.destroy_process_group()


def _run(world, steps, n_iter, bad):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, steps, n_iter, q, bad)) for r in range(world)]
    for p in procs:
        p.start()
    out = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return out


def test_two_ranks_shard_colourings_and_take_max_time():
    world, steps, n_iter = 2, 4, 16
    everything, tmax, check = _run(world, steps, n_iter, bad=False)
    cols = sorted(j for rk in everything for (a, n) in rk for j in range(a, a + n))
    assert cols == list(range(world * steps * n_iter))   # disjoint and complete
    assert tmax == pytest.approx(2.5)
    assert check == {"checked": 1, "equal": True, "colourings": world * steps * n_iter}


def test_replica_check_catches_a_rank_with_wrong_counts():
    _, _, check = _run(2, 2, 4, bad=True)
    assert check["checked"] == 1 and check["equal"] is False
