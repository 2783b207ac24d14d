"""The multi-GPU form of the benchmark is replicas only: each rank advances its own
instances, and only a barrier and a max over ranks of the timed region connect the
ranks.  That host-side logic runs here on CPU with the gloo backend and two ranks (no
GPU involved): the process group comes up from the environment, the barrier passes, the
timing reduction returns the slowest rank's time on every rank, ranks draw different
seeds, and the reference arm does no work on ranks other than 0."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_setup()
    assert (w, r, local) == (world, rank, rank) and dist.get_backend() == "gloo"
    bench.barrier(w)
    t = bench.max_over_ranks(1.0 + rank, w)
    defs = bench.batch_defs(4)
    seeds = [d["seed"] + (rank << 32) for d in defs]

    class A:
        gpus, steps, warmup = world, 2, 3
    ref = bench.run_reference(A, w, r) if rank != 0 else None
    out.put((rank, t, seeds, ref))
    dist.destroy_process_group()


def test_two_rank_replicas_on_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, s0, _), (r1, t1, s1, ref1) = res
    assert t0 == t1 == 2.0                  # the slowest rank's time everywhere
    assert not set(s0) & set(s1)            # independent instances per rank
    assert ref1 == 0                        # the reference arm is rank 0's alone
