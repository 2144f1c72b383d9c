"""The bench's multi-rank host logic on CPU with gloo (world size 2): each
rank gets its own query batch over the same mesh, the step time is the
slowest rank's, the job value counts every rank's queries, and the
reference arm runs on rank 0 only."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    args = bench._args_from([])
    args.queries = 4096
    c = bench._workload(args, rank)
    ms = bench._max_over_ranks(1.0 + rank, "cpu")
    ref = bench.run_reference(bench._args_from(["--impl", "reference", "--steps", "1", "--warmup", "0",
                                                "--queries", "512", "--gpus", str(world)]))
    out[rank] = dict(q=c["queries"][:4].copy(), V=c["V"][:4].copy(), ms=ms,
                     value=bench._job_value(ms, args.queries, world), ref=ref)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
        r0, r1 = out[0], out[1]
    assert r0["ms"] == r1["ms"] == 2.0
    assert r0["value"] == r1["value"] == 2 * 4096 / 2e-3
    assert np.array_equal(r0["V"], r1["V"])            # one mesh, replicated
    assert not np.array_equal(r0["q"], r1["q"])        # each rank its own batch
    assert r1["ref"] is None and r0["ref"]["impl"] == "reference"
    assert r0["ref"]["n_gpus"] == world
