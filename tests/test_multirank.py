"""Multi-rank host logic on CPU with gloo (world size 2).

* The bench: each rank gets its own query batch over the same mesh, the step
  time is the slowest rank's, the job value counts every rank's queries, and
  the reference arm runs on rank 0 only.
* A body split across ranks (Sec. 3.6: the outer LogSumExp of Eq. lse_full2
  and its gradient, Eq. dlse_full, are associative sums over the body's
  vertices): each rank forms its shard's partial (m, s, v, gp, gt) from the
  FP64 oracle's per-vertex values, the partials are all-gathered over gloo,
  and the library's host-only merge (sd_pose_merge) must give the oracle's
  single-shard constraint and pose gradient."""
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


def _oracle_partial(v, g, Y, alpha_q):
    """One shard's partial in FP64, in sd_pose_partial's layout."""
    t = -alpha_q * v
    m = t.max()
    e = np.exp(t - m)
    return np.concatenate([[m, e.sum(), (e * v).sum()], (e[:, None] * g).sum(0),
                           (e[:, None] * np.cross(Y, g)).sum(0)])


def _shard_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import torch

    import oracle
    import synth
    from oracle import pose as PO
    from paper_2108_10480_gb300 import pose as gp
    P = synth.points_on_sphere(600, seed=3) * 2.0
    V0, _ = synth.geodesic_icosphere(5)
    X0 = (V0.astype(np.float64) * np.array([0.6, 0.4, 0.3])).astype(np.float32)
    pose = np.array([0.3, -0.7, 0.9, 0.4, -0.2, 2.9])
    alpha, alpha_q = 20.0, 40.0
    sc = oracle.Scene(points=P)
    X = PO.place(X0, pose, "f64")
    v, g, _ = sc.brute(X, alpha, threads=1)
    Y = X0.astype(np.float64) @ PO.rotation(pose[:3]).T
    # uneven contiguous shards
    cut = [0, X0.shape[0] // 3, X0.shape[0]]
    a, b = cut[rank], cut[rank + 1]
    part = torch.from_numpy(_oracle_partial(v[a:b], g[a:b], Y[a:b], alpha_q))
    parts = [torch.empty_like(part) for _ in range(world)]
    dist.all_gather(parts, part)
    merged = gp.merge_partials(torch.stack(parts).numpy(), pose, alpha_q)
    D, G, _, _, _ = PO.pose_objective(sc, X0, pose, alpha, alpha_q, precision="f64", threads=1)
    out[rank] = dict(merged=merged, D=D, G=G, swapped=gp.merge_partials(torch.stack(parts[::-1]).numpy(), pose,
                                                                         alpha_q))
    dist.barrier()
    dist.destroy_process_group()


def test_body_split_across_two_ranks():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_shard_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
        r0, r1 = out[0], out[1]
    assert np.array_equal(r0["merged"], r1["merged"])
    for r in (r0, r1):
        assert abs(r["merged"][0] - r["D"]) <= 1e-12 * max(abs(r["D"]), 1.0)
        assert np.abs(r["merged"][1:] - r["G"]).max() <= 1e-12 * max(np.abs(r["G"]).max(), 1.0)
        assert np.abs(r["swapped"] - r["merged"]).max() <= 1e-13 * max(np.abs(r["merged"]).max(), 1.0)
