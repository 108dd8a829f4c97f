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


# --------------------------------------------------------------------------- exchange
def _exchange_workload():
    from paper_2511_16576_gb300 import synth
    return synth.Workload("exchange", 300, (8, 24), "uniform", (5e-3, 2e-2), 32, 8, 4, 20)


def _union(world):
    from paper_2511_16576_gb300 import dist as D
    from paper_2511_16576_gb300 import synth
    w0 = _exchange_workload()
    shards = [synth.make_database(D.shard_workload(w0, r)) for r in range(world)]
    xy = np.concatenate([s.xy for s in shards])
    offs = [np.zeros(1, np.int64)]
    base = 0
    for s in shards:
        offs.append(s.offsets[1:] + base)
        base += s.n_vertices
    union = synth.PolySet(xy, np.concatenate(offs), np.concatenate([s.centre for s in shards]),
                          np.concatenate([s.rbar for s in shards]))
    return w0, shards, union


def _oracle_search(orc, w, db, db_hashes, q_sig, q_xy, q_off, k):
    """Every bucket candidate refined exactly (no top-m cut): top-k by (J desc, id asc)."""
    rp, cand = orc.candidates(q_sig, db_hashes, w.bands, w.rows, w.T)
    Q = len(q_off) - 1
    ids = np.full((Q, k), -1, np.int64)
    jj = np.full((Q, k), -1.0)
    for q in range(Q):
        qp = q_xy[q_off[q]:q_off[q + 1]]
        c = cand[rp[q]:rp[q + 1]].astype(np.int64)
        j = np.array([orc.jaccard(qp, db.poly(int(i))) for i in c])
        pos = j > 0
        c, j = c[pos], j[pos]
        o = np.lexsort((c, -j))[:k]
        ids[q, :len(o)], jj[q, :len(o)] = c[o], j[o]
    return ids, jj


def _exchange_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2511_16576_gb300 import dist as D
    from paper_2511_16576_gb300 import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w0, shards, union = _union(world)
    db = shards[rank]
    h = oracle.sign(db.xy, db.offsets, w0.seed, w0.K, w0.T)
    # this rank's queries: perturbed copies of polygons of the whole database; rank 1 has none
    nq = 20 if rank == 0 else (0 if rank == 1 else 7)
    qs = synth.perturbed_queries(union, max(nq, 1), 500 + rank)
    if nq == 0:
        qs = synth.PolySet(np.zeros((0, 2), np.int32), np.zeros(1, np.int64),
                           np.zeros((0, 2), np.int64), np.zeros(0))
    q_sig = oracle.sign(qs.xy, qs.offsets, w0.seed, w0.K, w0.T) if qs.n else \
        np.zeros((0, w0.K), np.uint32)
    qb = D.QueryBatch(torch.from_numpy(q_sig.view(np.int32)), torch.from_numpy(qs.xy),
                      torch.from_numpy(qs.offsets))
    base = int(D.shard_offsets(db.n)[rank])

    def local(allq, k):
        ids, j = _oracle_search(oracle, w0, db, h, allq.sig.numpy().view(np.uint32),
                                allq.xy.numpy(), allq.offsets.numpy(), k)
        return torch.from_numpy(ids), torch.from_numpy(j)

    gid, gj = D.global_search(local, qb, base, 10)
    np.save(os.path.join(out_dir, f"ids{rank}.npy"), gid.numpy())
    np.save(os.path.join(out_dir, f"j{rank}.npy"), gj.numpy())
    np.save(os.path.join(out_dir, f"q{rank}.npy"), qs.xy)
    np.save(os.path.join(out_dir, f"qo{rank}.npy"), qs.offsets)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_search_equals_single_process_over_the_union(world):
    """The exchange (all-gather of queries, local search per shard, all-gather of the shard
    lists, merge by (J desc, global id asc)) returns, for every rank's queries, the top-10 a
    single process finds searching the union of the shards; one rank has no queries."""
    import oracle
    oracle.build()
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_exchange_main, args=(world, _free_port(), d), nprocs=world, join=True,
                           start_method="spawn")
        got = [(np.load(os.path.join(d, f"ids{r}.npy")), np.load(os.path.join(d, f"j{r}.npy")),
                np.load(os.path.join(d, f"q{r}.npy")), np.load(os.path.join(d, f"qo{r}.npy")))
               for r in range(world)]
    w0, _, union = _union(world)
    uh = oracle.sign(union.xy, union.offsets, w0.seed, w0.K, w0.T)
    found = mixed = 0
    for r, (ids, j, qxy, qoff) in enumerate(got):
        assert ids.shape == (len(qoff) - 1, 10)
        if len(qoff) == 1:
            continue
        q_sig = oracle.sign(qxy, qoff, w0.seed, w0.K, w0.T)
        ref_ids, ref_j = _oracle_search(oracle, w0, union, uh, q_sig, qxy, qoff, 10)
        assert np.array_equal(ids, ref_ids), r
        assert np.allclose(j, ref_j, rtol=0, atol=1e-15), r
        found += int((ids >= 0).sum())
        # queries whose top-10 holds polygons of more than one shard
        shard_of = np.where(ids >= 0, ids // w0.n_polys, -1)
        mixed += sum(len(set(row[row >= 0].tolist())) > 1 for row in shard_of)
    assert found > 0 and mixed > 0


def test_merge_topk_orders_and_pads():
    import torch

    from paper_2511_16576_gb300 import dist as D
    j_a = torch.tensor([[0.9, 0.5, -1.0], [0.3, -1.0, -1.0]], dtype=torch.float64)
    i_a = torch.tensor([[7, 3, -1], [2, -1, -1]])
    j_b = torch.tensor([[0.9, 0.6, 0.5], [-1.0, -1.0, -1.0]], dtype=torch.float64)
    i_b = torch.tensor([[4, 11, 1], [-1, -1, -1]])
    ids, j = D.merge_topk([j_a, j_b], [i_a, i_b], 4)
    # ties on J go to the smaller global id; empty slots pad with -1
    assert ids.tolist() == [[4, 7, 11, 1], [2, -1, -1, -1]]
    assert j.tolist() == [[0.9, 0.9, 0.6, 0.5], [0.3, -1.0, -1.0, -1.0]]
