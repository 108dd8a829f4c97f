"""Search-quality measurement: recall@k and queries/s of the plain and learned forms.

The paper evaluates PolyMinHash by Recall@k against the exact brute-force search and by
the time of hashmap lookup + refinement (Sec. 5.2, Table "Impact of MinHash lengths").
Here, on the GPU:

* brute force (the ground truth): every database polygon whose bounding box overlaps a
  query's (pmh_bbox_join), exact fp64 Jaccard of all those pairs (pmh_pair_jaccard),
  top-k by (J desc, id asc);
* the approximate search: sign the queries, join the buckets, count agreements, keep the
  top-m candidates -- by agreement count (plain form) or by the learned reranker's
  predicted Jaccard (learned form) -- and refine them exactly to the top-k;
* recall@k = |returned top-k among the exact top-k| / k (a returned polygon whose exact J
  ties the k-th exact J within 1e-9 also counts; if fewer than k polygons have J > 0 the
  denominator is that number).

Every step runs in the library's kernels; this module only orchestrates and times.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import binding as B


@dataclasses.dataclass
class Truth:
    ids: np.ndarray     # int32 [Q, k], -1 padded
    j: np.ndarray       # float64 [Q, k]
    n_pos: np.ndarray   # int [Q] number of polygons with J > 0 (capped at k)
    pairs: int          # exact Jaccard evaluations done by the brute force


def brute_force_topk(ctx: B.Context, qp: B.Polys, dbp: B.Polys, k: int = 10) -> Truth:
    row_ptr, cand = B.bbox_join(ctx, qp, dbp)
    Q = qp.n
    counts = (row_ptr[1:] - row_ptr[:-1]).cpu().numpy()
    qid = torch.repeat_interleave(torch.arange(Q, device=cand.device, dtype=torch.int32),
                                  torch.from_numpy(counts).to(cand.device))
    j = B.pair_jaccard(ctx, qp, dbp, qid, cand).cpu().numpy()
    rp = row_ptr.cpu().numpy()
    cd = cand.cpu().numpy()
    ids = np.full((Q, k), -1, np.int32)
    jj = np.full((Q, k), -1.0)
    n_pos = np.zeros(Q, np.int64)
    for q in range(Q):
        seg_j = j[rp[q]:rp[q + 1]]
        seg_i = cd[rp[q]:rp[q + 1]]
        pos = seg_j > 0
        seg_j, seg_i = seg_j[pos], seg_i[pos]
        order = np.lexsort((seg_i, -seg_j))[:k]
        ids[q, :len(order)] = seg_i[order]
        jj[q, :len(order)] = seg_j[order]
        n_pos[q] = len(order)
    return Truth(ids, jj, n_pos, int(len(cd)))


def recall_at_k(ann_ids: np.ndarray, ann_j: np.ndarray, truth: Truth, k: int = 10,
                tol: float = 1e-9) -> float:
    rec = []
    for q in range(len(truth.ids)):
        denom = int(truth.n_pos[q])
        if denom == 0:
            continue
        exact = set(int(x) for x in truth.ids[q, :denom])
        kth = truth.j[q, denom - 1] if denom == k else 0.0
        good = 0
        for i, jv in zip(ann_ids[q, :k], ann_j[q, :k]):
            if i < 0:
                continue
            if int(i) in exact or (denom == k and jv >= kth - tol and jv > 0):
                good += 1
        rec.append(min(good, denom) / denom)
    return float(np.mean(rec)) if rec else 1.0


@dataclasses.dataclass
class Searcher:
    """The approximate search over one database index.

    Plain form: bucket candidates -> agreement counts -> top-m by count -> exact top-k.
    Learned form: the top-`shortlist` candidates by count are rescored by the reranker and
    the top-m by predicted Jaccard are refined."""
    ctx: B.Context
    index: B.Index
    params: B.Params
    dbp: B.Polys
    dbh: torch.Tensor
    reranker: B.Reranker | None = None
    shortlist: int = 64

    def candidates(self, qp: B.Polys, stream=None):
        qh = B.minhash_sign(self.ctx, qp, self.params, stream=stream)
        row_ptr, cand = B.lsh_query(self.ctx, self.index, qh, stream=stream)
        count, _ = B.jaccard_estimate(self.ctx, qh, self.dbh, row_ptr, cand, self.params,
                                      bandmask=False, stream=stream)
        return qh, row_ptr, cand, count

    def shortlisted(self, qp: B.Polys, stream=None):
        """(qh, CSR of the count shortlist, its features, total bucket candidates)."""
        qh, row_ptr, cand, count = self.candidates(qp, stream)
        ids1, nn1 = B.topm(self.ctx, row_ptr, cand, count, self.shortlist, stream=stream)
        rp2, c2 = B.lists_to_csr(self.ctx, ids1, nn1, stream=stream)
        feat = B.rerank_features(self.ctx, qp, self.dbp, qh, self.dbh, rp2, c2, self.params,
                                 stream=stream)
        return qh, rp2, c2, feat, int(cand.numel())

    def query(self, qp: B.Polys, m: int, k: int = 10, learned: bool = False, stream=None):
        if learned:
            qh, rp2, c2, feat, ncand = self.shortlisted(qp, stream)
            score = self.reranker.forward(feat, stream=stream)
            ids, nn = B.topm(self.ctx, rp2, c2, None, m, score=score, stream=stream)
        else:
            qh, row_ptr, cand, count = self.candidates(qp, stream)
            ncand = int(cand.numel())
            ids, nn = B.topm(self.ctx, row_ptr, cand, count, m, stream=stream)
        top_ids, top_j = B.refine_topk(self.ctx, qp, self.dbp, ids, nn, min(k, m), stream=stream)
        return top_ids, top_j, ncand


def training_pairs(ctx: B.Context, searcher: Searcher, tp: B.Polys):
    """Features and exact-Jaccard labels of the shortlisted candidates of training queries."""
    qh, rp2, c2, feat, _ = searcher.shortlisted(tp)
    E = int(rp2[-1].item())
    c2 = c2[:E]
    counts = rp2[1:] - rp2[:-1]
    qid = torch.repeat_interleave(torch.arange(tp.n, device=c2.device, dtype=torch.int32), counts)
    label = B.pair_jaccard(ctx, tp, searcher.dbp, qid, c2).to(torch.float32)
    return feat[:E].contiguous(), label


def train_reranker(reranker: B.Reranker, feat: torch.Tensor, label: torch.Tensor, epochs: int = 8,
                   batch: int = 4096, lr: float = 2e-3, seed: int = 0):
    """Minibatch Adam on the GPU; returns the mean loss of each epoch."""
    g = torch.Generator(device=feat.device)
    g.manual_seed(seed)
    n = feat.shape[0]
    losses = []
    for _ in range(epochs):
        perm = torch.randperm(n, generator=g, device=feat.device)
        tot = torch.zeros((), device=feat.device)
        nb = 0
        for s in range(0, n, batch):
            idx = perm[s:s + batch]
            tot += reranker.train_step(feat[idx].contiguous(), label[idx].contiguous(), lr)[0]
            nb += 1
        losses.append(float(tot.item()) / max(nb, 1))
    return losses


def timed(fn, stream=None):
    stream = stream or torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return out, e0.elapsed_time(e1) * 1e-3


def sweep(searcher: Searcher, qp: B.Polys, truth: Truth, n_eval: int, ms=(8, 10, 12, 16, 24, 32, 64),
          k: int = 10, learned: bool = False):
    """recall@k (first n_eval queries) and queries/s (whole batch) for each m."""
    rows = []
    for m in ms:
        searcher.query(qp, m, k, learned)  # warm-up
        (ids, j, ncand), t = timed(lambda: searcher.query(qp, m, k, learned))
        r = recall_at_k(ids.cpu().numpy()[:n_eval], j.cpu().numpy()[:n_eval], truth, k)
        rows.append({"m": m, "recall": r, "qps": qp.n / t, "seconds": t,
                     "candidates_per_query": ncand / qp.n})
    return rows


def best_at_recall(rows, target: float = 0.9):
    ok = [r for r in rows if r["recall"] >= target]
    return max(ok, key=lambda r: r["qps"]) if ok else None


# ----------------------------------------------------------------------------
# The batched search: queries in fixed-size batches through a captured graph (A9)
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Batches:
    """A query set cut into batches of at most `size` polygons (device tensors, offsets
    rebased per batch), with the largest batch's vertex count."""
    xy: list
    off: list
    n: list
    size: int
    max_vertices: int

    @property
    def total(self) -> int:
        return int(sum(self.n))


def make_batches(xy: torch.Tensor, offsets: np.ndarray, size: int, pinned: bool = False) -> Batches:
    """Cut a query set (xy on the device or pinned host, offsets on the host) into batches."""
    offsets = np.asarray(offsets, np.int64)
    Q = len(offsets) - 1
    xs, os_, ns = [], [], []
    vmax = 3
    for q0 in range(0, Q, size):
        q1 = min(Q, q0 + size)
        b, e = int(offsets[q0]), int(offsets[q1])
        o = torch.from_numpy(offsets[q0:q1 + 1] - b)
        o = o.pin_memory() if pinned else o.to(xy.device)
        xs.append(xy[b:e])
        os_.append(o)
        ns.append(q1 - q0)
        vmax = max(vmax, e - b)
    return Batches(xs, os_, ns, size, vmax)


def batch_capacity(ctx: B.Context, index: B.Index, params: B.Params, qp: B.Polys, size: int) -> int:
    """Largest candidate total of any batch of `size` consecutive queries (plus a margin)."""
    qh = B.minhash_sign(ctx, qp, params)
    row_ptr, _ = B.lsh_query(ctx, index, qh)
    rp = row_ptr.cpu().numpy()
    ends = np.minimum(np.arange(0, qp.n, size) + size, qp.n)
    per = rp[ends] - rp[np.arange(0, qp.n, size)]
    return int(max(per.max() if len(per) else 1, 1) * 1.25) + 1024


def run_batches(g: B.QueryGraph, batches: Batches, ids_out: torch.Tensor, j_out: torch.Tensor | None,
                stream=None):
    """Replay the graph on every batch; the refined top-k of batch b (or, for a graph
    without refinement, its top-m lists, with j_out None) go to its rows of ids_out /
    j_out (device or pinned host tensors, copied on the graph's stream)."""
    q0 = 0
    for xy, off, n in zip(batches.xy, batches.off, batches.n):
        g.run(xy, off, stream=stream)
        if g.k > 0:
            ids_out[q0:q0 + n].copy_(g.ref_ids[:n], non_blocking=True)
            j_out[q0:q0 + n].copy_(g.ref_j[:n], non_blocking=True)
        else:
            ids_out[q0:q0 + n].copy_(g.top_ids[:n], non_blocking=True)
        q0 += n


def graph_sweep(ctx: B.Context, index: B.Index, dbp: B.Polys, batches: Batches, cap: int,
                truth: Truth, n_eval: int, ms, k: int = 10, rerank: B.Reranker | None = None,
                shortlist: int = 64):
    """recall@k (first n_eval queries) and queries/s (all batches, graph replays) per m."""
    dev = torch.device("cuda", ctx.device)
    Q = batches.total
    ids = torch.empty((Q, k), dtype=torch.int32, device=dev)
    jj = torch.empty((Q, k), dtype=torch.float64, device=dev)
    rows = []
    for m in ms:
        g = B.QueryGraph(ctx, index, batches.size, batches.max_vertices, cap, m, db=dbp, k=k,
                         rerank=rerank, shortlist=max(shortlist, m))
        try:
            run_batches(g, batches, ids, jj)     # warm-up
            flags = g.status()[0]
            _, t = timed(lambda: run_batches(g, batches, ids, jj))
        finally:
            g.close()
        r = recall_at_k(ids.cpu().numpy()[:n_eval], jj.cpu().numpy()[:n_eval], truth, k)
        rows.append({"m": m, "recall": r, "qps": Q / t, "seconds": t, "flags": flags})
    return rows


def batch_size_sweep(ctx: B.Context, index: B.Index, params: B.Params, dbp: B.Polys,
                     dbh: torch.Tensor, qs_xy: torch.Tensor, qs_offsets: np.ndarray,
                     sizes=(1, 64, 1024, 4096), m: int = 32, k: int = 10,
                     queries_per_size: int = 4096, rerank: B.Reranker | None = None,
                     shortlist: int = 64):
    """Per batch size: queries/s and mean milliseconds per batch of the captured graph
    (replays, inputs on the device) beside the same steps as plain library calls (upload,
    sign, join, agreement, top-m by count, refinement: several launches and host
    synchronisations per batch), over the first `queries_per_size` queries."""
    out = []
    for size in sizes:
        n_q = min(queries_per_size, len(qs_offsets) - 1)
        n_q -= n_q % size if n_q >= size else 0
        if n_q == 0:
            continue
        batches = make_batches(qs_xy, qs_offsets[:n_q + 1], size)
        qp = B.poly_upload(ctx, qs_xy[:int(qs_offsets[n_q])], torch.from_numpy(qs_offsets[:n_q + 1]).to(qs_xy.device))
        cap = batch_capacity(ctx, index, params, qp, size)
        qp.close()
        g = B.QueryGraph(ctx, index, size, batches.max_vertices, cap, m, db=dbp, k=k, rerank=rerank,
                         shortlist=max(shortlist, m))
        dev = qs_xy.device
        ids = torch.empty((n_q, k if k > 0 else m), dtype=torch.int32, device=dev)
        jj = torch.empty((n_q, k), dtype=torch.float64, device=dev) if k > 0 else None
        run_batches(g, batches, ids, jj)
        _, t_graph = timed(lambda: run_batches(g, batches, ids, jj))
        g.close()

        def plain():
            for xy, off, n in zip(batches.xy, batches.off, batches.n):
                qp = B.poly_upload(ctx, xy, off)
                qh = B.minhash_sign(ctx, qp, params)
                row_ptr, cand = B.lsh_query(ctx, index, qh)
                count, _ = B.jaccard_estimate(ctx, qh, dbh, row_ptr, cand, params, bandmask=False)
                tid, tn = B.topm(ctx, row_ptr, cand, count, m)
                if k > 0:
                    B.refine_topk(ctx, qp, dbp, tid, tn, k)
                qp.close()
        plain()
        _, t_plain = timed(plain)
        out.append({"batch": size, "queries": n_q, "graph_qps": n_q / t_graph,
                    "graph_ms_per_batch": 1e3 * t_graph / len(batches.n),
                    "plain_calls_qps": n_q / t_plain,
                    "plain_calls_ms_per_batch": 1e3 * t_plain / len(batches.n)})
    return out
