"""The multi-process (replica) path of bench.py on CPU: two gloo ranks set up
the process group from the launcher's environment, meet at barriers and
take the max of their timings, as the N-GPU run does over NCCL.  The stencil
path itself does not shard (each problem runs on one GPU), so this is the
only cross-rank exchange."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import torch.distributed as dist

    import bench

    r, w, local = bench.dist_setup(world)
    assert (r, w, local) == (rank, world, rank)
    bench.barrier(w)
    got = bench.allreduce_max(10.0 + rank, w)
    bench.barrier(w)
    out[rank] = got
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_max_timing():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    assert dict(out) == {0: 11.0, 1: 11.0}


def test_single_process_needs_no_group():
    import bench
    assert bench.allreduce_max(3.5, 1) == 3.5
    bench.barrier(1)
