"""The multi-rank host path on CPU: two gloo ranks shard the workload, time their step and
take the maximum over ranks; the union of the shards' signatures is what one process
computing both shards gets (independent shards, no data-path collective)."""
import os
import socket
import tempfile

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import time

    import torch.distributed as dist

    import oracle
    from paper_2511_16576_gb300 import dist as D
    from paper_2511_16576_gb300 import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w0 = synth.Workload("tiny", 40, (8, 24), "uniform", (1e-2, 3e-2), 16, 4, 4, 5)
    w, r = D.shard_workload(w0, D.env()[1]), D.env()[1]
    db = synth.make_database(w)
    dist.barrier()
    t0 = time.perf_counter()
    h = oracle.sign(db.xy, db.offsets, w.seed, w.K, w.T)
    dt = time.perf_counter() - t0 + 0.01 * r          # rank 1 is made the slower one
    dist.barrier()
    worst = D.max_over_ranks(dt)
    np.save(os.path.join(out_dir, f"h{r}.npy"), h)
    np.save(os.path.join(out_dir, f"t{r}.npy"), np.array([dt, worst]))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_time():
    import oracle
    from paper_2511_16576_gb300 import dist as D
    from paper_2511_16576_gb300 import synth
    oracle.build()
    world = 2
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank_main, args=(world, _free_port(), d), nprocs=world, join=True,
                           start_method="spawn")
        t = [np.load(os.path.join(d, f"t{r}.npy")) for r in range(world)]
        h = [np.load(os.path.join(d, f"h{r}.npy")) for r in range(world)]
    # every rank sees the same maximum, and it is the slowest rank's time
    assert t[0][1] == t[1][1] == max(t[0][0], t[1][0])
    # the shards differ (different generator seeds) and each equals a single-process run
    w0 = synth.Workload("tiny", 40, (8, 24), "uniform", (1e-2, 3e-2), 16, 4, 4, 5)
    for r in range(world):
        w = D.shard_workload(w0, r)
        db = synth.make_database(w)
        assert np.array_equal(h[r], oracle.sign(db.xy, db.offsets, w.seed, w.K, w.T))
    assert not np.array_equal(h[0], h[1])
    assert D.job_throughput(40 * 16, world, 0.5) == 2 * 40 * 16 / 0.5


def test_single_process_defaults():
    from paper_2511_16576_gb300 import dist as D
    assert D.env()[0] >= 1
    assert D.max_over_ranks(3.5) == 3.5
