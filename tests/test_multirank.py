"""The multi-GPU path of bench.py on CPU: world_size 2 over gloo.

Each rank holds a replica of the index and answers its own query batches;
the only collective is the timing/work reduction (max of times, sum of work).
Here the ranks answer their batches with the CPU oracle, so the sharding and
reduction logic run without a GPU."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist

    import bench
    import synth
    from oracle.oracle import Oracle

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    w = synth.make("genome", 0.005, m=1 << 14)
    batches = bench.extra_batches(w, 2, rank)
    o = Oracle(w.K, w.B, w.R, w.m, w.eta, w.seed)
    o.insert_seq_batch(w.sets.ids, w.sets.data, w.sets.offsets, 31)
    keys = 0
    answers = []
    for q in batches:
        ids, off = o.query_batch("seq", q.data, q.offsets, 31)
        answers.append((ids, off))
        keys += bench.keys_in(q, 31)
    fake_ms = 10.0 * (rank + 1)
    (t_max,), (k_sum,) = bench.reduce_over_ranks(dist, [fake_ms], [keys], "cpu")
    np.savez(out_path, keys=keys, t_max=t_max, k_sum=k_sum,
             first_batch=batches[0].data[:200], n_results=sum(int(a[1][-1]) for a in answers))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_batches_and_reduce(tmp_path):
    import torch.multiprocessing as mp

    port = _free_port()
    paths = [str(tmp_path / f"r{r}.npz") for r in range(2)]
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, paths[r])) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    r0, r1 = (np.load(p) for p in paths)
    # disjoint work: the ranks' batches differ
    assert not np.array_equal(r0["first_batch"], r1["first_batch"])
    # whole-job figures: time is the slowest rank's, work is the sum
    assert float(r0["t_max"]) == float(r1["t_max"]) == 20.0
    assert float(r0["k_sum"]) == float(r1["k_sum"]) == float(r0["keys"]) + float(r1["keys"])
    assert int(r0["n_results"]) > 0 and int(r1["n_results"]) > 0


def test_single_process_reduction_is_identity():
    import bench

    assert bench.reduce_over_ranks(None, [3.0, 4.0], [5, 6], "cpu") == ([3.0, 4.0], [5.0, 6.0])
