"""PolyMinHash benchmark: one step = one pass of the whole signature path over one batch.

Step (inputs resident in HBM when the timed region starts): the database polygons are
loaded into the library's polygon set and prepared (A0: validation, boxes, areas, y-slab
lists, signing plan), signed (A1: one persistent launch of the unified kernel through the
stream index), their band keys and bucket index rebuilt (A2, A3); then the query set runs
in batches of 4,096 through the captured query graph (A9): prep, signing, bucket join
(A4), agreement (A5), a shortlist by agreement count rescored by the learned reranker
(A7) to the top-m (A6), and exact fp64 refinement to the top-10 (A8).  Default workload:
the combined configuration -- 10,000,000 star / fractal polygons with 8-1,024 vertices
(16.7 GB of int32 vertices), area fractions log-uniform 1e-5..1e-2, K = 128, 16 bands x 8
rows, 100,000 perturbed-copy queries -- synthetic and seeded.

value = (N + Q) * K polygon-hashes per second of step time.  `e2e` is the same step
from pinned HOST buffers (the database and every query batch copied to the device, the
refined top-10 of every batch copied back, inside the timed region).  `roofline` is the
dominant kernel (the signing launch) against the measured integer-ALU peak, with its L2
and DRAM traffic from the committed ncu summary of the same kernel source.
`search` (after the timed region) is queries/s at recall@10 >= 0.9 of the plain
(agreement-count) and learned (reranker) forms, both through the graph, over band shapes.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Algorithmic 32-bit integer operations of the signing kernel, per unit of work it
# reports (pmh_sign_work):
#  walked stream point: 64-bit counter add (2), two xor-shift rounds (4 + 4), two
#    low-64-bit 64x64 multiplies (4 + 4), final xor-shift of the low word (2), field
#    extraction and half-open bbox test (6) = 26;
#  grid cell read by the indexed form: two offsets and the cell address = 8;
#  stream-index entry read: index and point loads, limit compare, bbox test = 10;
#  bbox candidate classified = 6;
#  polygon edge tested: straddle test (3), two 32x32->64 products (4), difference (2),
#    sign test and parity (3) = 12;
#  candidate decided by the coverage mask: cell address and code lookup = 6.
SIGN_OP_WEIGHTS = {"walk_points": 26, "cells": 8, "index_entries": 10, "candidates": 6,
                   "edge_tests": 12, "mask_decisions": 6}
# the signing kernel's sources: a profile summary applies only to the source it was taken on
SIGN_SOURCES = ["paper_2511_16576_gb300/csrc/sign_unified.cu",
                "paper_2511_16576_gb300/csrc/sign_common.cuh",
                "paper_2511_16576_gb300/csrc/pmh_internal.cuh"]
SIGN_PROFILE = "profiles/sign_unified_kernel_combined.md"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="combined")
    ap.add_argument("--n-polys", type=int, default=None, help="override database size")
    ap.add_argument("--n-queries", type=int, default=None)
    ap.add_argument("--batch", type=int, default=4096, help="queries per graph replay")
    ap.add_argument("--topm", type=int, default=32, help="candidates refined per query")
    ap.add_argument("--refine-k", type=int, default=10,
                    help="exact top-k of the refinement (0: the query graph stops at the top-m)")
    ap.add_argument("--shortlist", type=int, default=64, help="learned form: count shortlist")
    ap.add_argument("--search-shortlist", type=int, default=32,
                    help="learned form in the recall / queries-per-s sweep: count shortlist")
    ap.add_argument("--plain", action="store_true", help="time the plain form (no reranker)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=None, help="polygons in the CPU sample")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default sign variant")
    ap.add_argument("--no-search", action="store_true", help="skip the recall / queries-per-s sweep")
    ap.add_argument("--no-stream-index", action="store_true",
                    help="sign by walking every stream point (no stream index)")
    ap.add_argument("--cuda-profiler-range", action="store_true",
                    help="bracket the device-input timed steps with cudaProfilerStart/Stop (for "
                         "ncu --profile-from-start off)")
    ap.add_argument("--eval-queries", type=int, default=1000,
                    help="queries whose recall@10 is checked against brute force")
    ap.add_argument("--search-queries", type=int, default=5 * 4096,
                    help="queries whose graph replays time the search's queries/s")
    ap.add_argument("--search-max-candidates", type=float, default=5000.0,
                    help="skip a band shape with more bucket candidates per query than this")
    ap.add_argument("--train-queries", type=int, default=24000,
                    help="training queries of the search's reranker (x --shortlist pairs: ~1M)")
    ap.add_argument("--paper-sweep", action="store_true",
                    help="paper-shaped centred sets, one hashmap keyed on m = 1..5 hashes (prints one "
                         "JSON line with the table instead of the benchmark line)")
    ap.add_argument("--paper-scale", type=float, default=1.0, help="fraction of the paper set sizes")
    ap.add_argument("--paper-sets", default="n9,n12,n95",
                    help="paper-shaped sets of the sweep (n319 needs an exhaustive search over "
                         "319-vertex pairs: run it with --paper-scale)")
    return ap.parse_args()


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if sm:
            out = {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


def dist_setup(args):
    from paper_2511_16576_gb300 import dist as D
    return D.env()


def algorithmic_points(hashes_np: np.ndarray, T: int) -> int:
    """Stream points the definition examines: h + 1 for a hit, T for the sentinel."""
    h = hashes_np.astype(np.int64)
    return int(np.where(h < T, h + 1, T).sum())


def paper_sweep(args):
    """The paper's own configuration on paper-shaped sets (Sec. 3.1 centring and global MBR,
    Sec. 5.2-5.3 single hashmap keyed on the m-hash code, every candidate refined): per set
    and m = 1..5, the time to hash the database, to build and query the hashmap, to refine
    all candidates exactly, the candidates per query (pruning) and recall@10 against the
    exhaustive exact search over all polygons (they all overlap once centred)."""
    import torch
    from paper_2511_16576_gb300 import binding as B, synth, build as cuda_build
    from paper_2511_16576_gb300 import evaluate as ev
    cuda_build.build()
    dev = torch.device("cuda", 0)
    ctx = B.Context(0)
    stream = torch.cuda.current_stream()
    n_q, k = 100, 10

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1)

    def top_k(qn, row_ptr, cand, j):
        ids = np.full((qn, k), -1, np.int32)
        jj = np.full((qn, k), -1.0)
        n_pos = np.zeros(qn, np.int64)
        rp = row_ptr.cpu().numpy()
        cd = cand.cpu().numpy()
        jv = j.cpu().numpy()
        for q in range(qn):
            sj, si = jv[rp[q]:rp[q + 1]], cd[rp[q]:rp[q + 1]]
            pos = sj > 0
            sj, si = sj[pos], si[pos]
            o = np.lexsort((si, -sj))[:k]
            ids[q, :len(o)], jj[q, :len(o)], n_pos[q] = si[o], sj[o], len(o)
        return ids, jj, n_pos

    def truth_top_k(qn, jv, n):
        # exhaustive search: the 32 best of each query's row on the device, then the
        # (J desc, id asc) order of those on the host
        vals, idx = torch.topk(jv.view(qn, n), min(32, n), dim=1)
        vals, idx = vals.cpu().numpy(), idx.cpu().numpy().astype(np.int32)
        ids = np.full((qn, k), -1, np.int32)
        jj = np.full((qn, k), -1.0)
        n_pos = np.zeros(qn, np.int64)
        for q in range(qn):
            pos = vals[q] > 0
            sj, si = vals[q][pos], idx[q][pos]
            o = np.lexsort((si, -sj))[:k]
            ids[q, :len(o)], jj[q, :len(o)], n_pos[q] = si[o], sj[o], len(o)
        return ids, jj, n_pos

    rows = []
    for name in args.paper_sets.split(","):
        n_full, mean_v = synth.PAPER_SETS[name]
        n = max(1000, int(n_full * args.paper_scale))
        db = synth.paper_shaped(n, mean_v, seed=7 + len(rows))
        qs = synth.paper_queries(db, n_q, seed=107 + len(rows))
        dbp = B.poly_upload(ctx, torch.from_numpy(db.xy).to(dev), torch.from_numpy(db.offsets).to(dev))
        qp = B.poly_upload(ctx, torch.from_numpy(qs.xy).to(dev), torch.from_numpy(qs.offsets).to(dev))
        # exhaustive exact search: every (query, polygon) pair, in chunks of queries
        all_ids = torch.arange(db.n, dtype=torch.int32, device=dev)
        t_ids, t_j, t_pos = [], [], []
        bf_ms = 0.0
        for q0 in range(0, n_q, 10):
            qn = min(10, n_q - q0)
            qid = torch.arange(q0, q0 + qn, dtype=torch.int32, device=dev).repeat_interleave(db.n)
            cand = all_ids.repeat(qn)
            jv, ms = timed(lambda: B.pair_jaccard(ctx, qp, dbp, qid, cand))
            bf_ms += ms
            a, b_, c_ = truth_top_k(qn, jv, db.n)
            t_ids.append(a), t_j.append(b_), t_pos.append(c_)
        truth = ev.Truth(np.concatenate(t_ids), np.concatenate(t_j), np.concatenate(t_pos), n_q * db.n)
        for m in range(1, 6):
            P = B.make_params(m, 1, 1 << 24, flags=B.FLAG_STREAM_INDEX)
            B.minhash_sign(ctx, dbp, P)                       # builds the stream index for (seed, m)
            h, hash_ms = timed(lambda: B.minhash_sign(ctx, dbp, P))
            qh = B.minhash_sign(ctx, qp, P)

            def hashmap():
                index = B.lsh_build(ctx, h, P)
                rp, cd = B.lsh_query(ctx, index, qh)
                return index, rp, cd
            (index, row_ptr, cand), map_ms = timed(hashmap)
            index.close()
            counts = (row_ptr[1:] - row_ptr[:-1])
            qid = torch.repeat_interleave(torch.arange(n_q, dtype=torch.int32, device=dev), counts)
            E = int(row_ptr[-1].item())
            jv, ref_ms = timed(lambda: B.pair_jaccard(ctx, qp, dbp, qid, cand[:E]) if E else
                               torch.zeros(0, dtype=torch.float64, device=dev))
            ids, jj, _ = top_k(n_q, row_ptr, cand[:E], jv)
            rows.append({"set": name, "polygons": db.n, "mean_vertices": db.n_vertices / db.n, "m": m,
                         "hash_ms": hash_ms, "hashmap_ms": map_ms, "refine_ms": ref_ms,
                         "candidates_per_query": E / n_q, "pruning": 1.0 - E / (n_q * db.n),
                         "recall_at_10": ev.recall_at_k(ids, jj, truth, k),
                         "brute_force_ms": bf_ms})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
        qp.close()
        dbp.close()
    print(json.dumps({"paper_sweep": rows, "queries": n_q, "k": k, "scale": args.paper_scale}), flush=True)
    ctx.close()


def nominal_int_peak(dev, clk):
    """SMs x 128 integer lanes x the maximum SM clock, in T int-op/s (None if unknown)."""
    try:
        import torch
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = float(clk.get("sm_max_mhz") or 0.0) if isinstance(clk, dict) else 0.0
        return sms * 128 * mhz * 1e6 / 1e12 if mhz > 0 else None
    except Exception:  # measurement context only: never fail the benchmark line for it
        return None


def hbm_peak_gbs():
    """Measured HBM copy bandwidth of this GPU pool (GB/s), if the peaks file is present."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    for key in ("hbm_gbs", "hbm_GBps", "hbm"):
        if isinstance(d.get(key), (int, float)):
            return float(d[key])
    return None


def arm_config(args, w, db, Q, world):
    """The workload both arms report (the reference arm runs a sample of it)."""
    return {"workload": f"{w.name}: {db.n} {'fractal ' if w.fractal else ''}star polygons "
                        f"({db.n_vertices} vertices, {w.n_range[0]}-{w.n_range[1]} per polygon), "
                        f"K={w.K}, {w.bands}x{w.rows} bands, {Q} perturbed-copy queries in batches of "
                        f"{args.batch}, {'plain' if args.plain else 'learned'} top-{args.topm} "
                        + (f"refined to top-{args.refine_k}" if args.refine_k > 0 else "lists (no refinement)"),
            "l2": (f"inputs larger than L2 ({db.xy.nbytes / 1e6:.0f} MB of vertices)"
                   if db.xy.nbytes > 129e6 else
                   f"inputs smaller than L2 ({db.xy.nbytes / 1e6:.0f} MB of vertices), L2 not flushed"),
            "parallelism": f"{world} shard(s), one exchange of the query batches" if world > 1
            else "1 GPU"}


def run_reference(args, w):
    """The oracle as it stands, on the host cores, on a bounded sample of the workload."""
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    import oracle
    from paper_2511_16576_gb300 import synth
    oracle.build()
    n_sample = args.cpu_sample or 2000
    db = synth.make_database(w, args.n_polys)
    rng = np.random.default_rng(7)
    cores = os.cpu_count() or 1
    times = []
    for step in range(args.warmup + args.steps):
        ids = np.sort(rng.choice(db.n, n_sample, replace=False))
        sub = db.subset(ids)
        t0 = time.perf_counter()
        h = oracle.sign(sub.xy, sub.offsets, w.seed, w.K, w.T, nthreads=cores)
        oracle.band_keys(h, w.bands, w.rows, w.T, w.lsh_seed)
        t1 = time.perf_counter()
        if step >= args.warmup:
            times.append(t1 - t0)
    t = float(np.mean(times))
    value = n_sample * w.K / t
    line = {
        "impl": "reference", "metric": "polygon-hashes/s (N*K/s)", "value": value,
        "unit": "hashes/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": arm_config(args, w, db, args.n_queries or w.n_queries, world),
        "cpu_baseline": {"value": value, "unit": "hashes/s", "cores": cores, "kind": "oracle",
                         "sample": f"oracle sign + band keys of {n_sample} random polygons of the "
                                   f"{w.n_polys}-polygon workload per step"},
        "e2e": {"value": value, "unit": "hashes/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(w, db, seconds_target=15.0, n_sample=None):
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(11)
    n = n_sample or 256
    # grow the sample until it takes a few seconds, then size it for the target
    while True:
        ids = np.sort(rng.choice(db.n, min(n, db.n), replace=False))
        sub = db.subset(ids)
        t0 = time.perf_counter()
        oracle.sign(sub.xy, sub.offsets, w.seed, w.K, w.T, nthreads=cores)
        dt = time.perf_counter() - t0
        if n_sample or dt > 2.0 or n >= db.n:
            break
        n = min(db.n, int(n * max(2.0, min(8.0, seconds_target / 4 / max(dt, 1e-3)))))
    return {"value": len(ids) * w.K / dt, "unit": "hashes/s", "cores": cores, "kind": "oracle",
            "sample": f"oracle sign of {len(ids)} random polygons x K={w.K} of the "
                      f"{db.n}-polygon workload ({dt:.1f} s, {cores} threads)"}


def sources_sha(paths) -> str:
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def read_profile(path: str) -> dict:
    """`key: value` lines of a committed ncu summary (empty if absent)."""
    out = {}
    try:
        with open(os.path.join(ROOT, path)) as f:
            for line in f:
                line = line.strip().lstrip("-* ").strip("`")
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    out[k.strip()] = v.strip()
    except OSError:
        pass
    return out


def profiled_counters(polys_in_launch: int, workload: str) -> dict | None:
    """DRAM and L2 bytes and instructions per launch of the signing kernel, from the ncu
    summary taken on this same kernel source and workload (scaled by polygons to this
    launch), else None."""
    p = read_profile(SIGN_PROFILE)
    if not p or p.get("source_sha") != sources_sha(SIGN_SOURCES):
        return None
    if not str(p.get("workload", "")).startswith(workload):
        return None
    try:
        scale = polys_in_launch / float(p["launch_polygons"])
        return {"dram_bytes": float(p["dram_bytes"]) * scale, "lts_bytes": float(p["lts_bytes"]) * scale,
                "inst_executed": float(p["inst_executed"]) * scale,
                "l2_throughput_pct": float(p["l2_throughput_pct"]),
                "dram_throughput_pct": float(p["dram_throughput_pct"]),
                "captured_on": p.get("workload"), "scale": scale}
    except (KeyError, ValueError):
        return None


def search_quality(args, w, B, ctx, db, qs, h, dbp, q_xy, q_off, P):
    """queries/s at recall@10 >= 0.9 of the plain (agreement count) and learned (reranker)
    forms, both through the captured query graph in batches (after the timed region).

    The database signatures are indexed with 64 x 2, 32 x 4 and the workload's 16 x 8
    bands (short bands make more polygons candidates); for each shape the top-m sweep gives
    recall@10 on the first eval queries (ground truth: the GPU brute force -- every
    box-overlapping polygon, exact fp64 Jaccard) and queries/s over all queries; the
    reranker is trained on the shortlists of separate training queries (GPU kernels, Adam)
    for each shape.  The best queries/s reaching recall 0.9 is reported per form."""
    import torch
    from paper_2511_16576_gb300 import evaluate as ev
    from paper_2511_16576_gb300 import synth
    dev = q_xy.device
    n_eval = min(args.eval_queries, qs.n)
    qe = qs.subset(np.arange(n_eval))
    qep = B.poly_upload(ctx, torch.from_numpy(qe.xy).to(dev), torch.from_numpy(qe.offsets).to(dev))
    truth, t_bf = ev.timed(lambda: ev.brute_force_topk(ctx, qep, dbp, 10))
    qep.close()
    n_s = min(qs.n, max(args.search_queries, n_eval))
    qp = B.poly_upload(ctx, q_xy[:int(qs.offsets[n_s])], q_off[:n_s + 1])
    batches = ev.make_batches(q_xy, qs.offsets[:n_s + 1], args.batch)
    tq = synth.perturbed_queries(db, args.train_queries, w.query_seed + 1000)
    tp = B.poly_upload(ctx, torch.from_numpy(tq.xy).to(dev), torch.from_numpy(tq.offsets).to(dev))
    out = {"eval_queries": n_eval, "timed_queries": n_s, "batch": args.batch, "k": 10,
           "target_recall": 0.9, "bf_pairs_per_query": truth.pairs / n_eval,
           "bf_seconds_eval_queries": t_bf, "forms": {}}
    ms = tuple(range(10, 25)) + (28, 32)   # refined to the top-10: m >= 10; every m to 24
    shapes = [b for b in (w.K // 2, w.K // 4, w.bands) if b >= 1 and w.K % b == 0]
    for bands in dict.fromkeys(shapes):
        params = B.make_params(w.K, bands, w.T, w.seed, w.lsh_seed, P.flags)
        index = B.lsh_build(ctx, h, params)
        cap = ev.batch_capacity(ctx, index, params, qp, args.batch)
        key = f"{params.bands}x{params.rows}"
        if cap / args.batch > args.search_max_candidates * 1.25:
            out["forms"][key] = {"bands": key, "skipped": f"{cap / args.batch / 1.25:.0f} bucket candidates "
                                 f"per query in the largest batch (> {args.search_max_candidates:.0f})"}
            index.close()
            continue
        plain = ev.graph_sweep(ctx, index, dbp, batches, cap, truth, n_eval, ms)
        # trained on the wider count shortlist (more pairs per training query), used on the
        # search's own
        s = ev.Searcher(ctx, index, params, dbp, h, shortlist=max(args.shortlist, args.search_shortlist))
        feat, lab = ev.training_pairs(ctx, s, tp)
        rr = B.Reranker(ctx, seed=1)
        # 24 epochs at the default rate, then 8 at a quarter of it (the same Adam moments)
        (losses, t_train) = ev.timed(lambda: ev.train_reranker(rr, feat, lab, epochs=24) +
                                     ev.train_reranker(rr, feat, lab, epochs=8, lr=5e-4, seed=1))
        learned = ev.graph_sweep(ctx, index, dbp, batches, cap, truth, n_eval, ms, rerank=rr,
                                 shortlist=args.search_shortlist)
        rr.close()
        out["forms"][key] = {"bands": key, "candidates_per_query_cap": cap / args.batch,
                             "plain_curve": plain, "plain": ev.best_at_recall(plain),
                             "learned_curve": learned, "learned": ev.best_at_recall(learned),
                             "train_pairs": int(feat.shape[0]), "train_loss_per_epoch": losses,
                             "train_seconds": t_train}
        del feat, lab
        index.close()
    tp.close()
    qp.close()
    for form in ("plain", "learned"):
        best = [(f[form], k) for k, f in out["forms"].items() if f.get(form)]
        if best:
            r, k = max(best, key=lambda t: t[0]["qps"])
            out[form] = {"bands": k, **r}
        else:
            out[form] = None
    if out["plain"] and out["learned"]:
        out["learned_over_plain_qps"] = out["learned"]["qps"] / out["plain"]["qps"]
    return out


def train_for_step(args, w, B, ctx, db, dbp, h, index, P):
    """The reranker of the timed step: trained (untimed) on the shortlists of separate
    training queries at the step's own banding."""
    import torch
    from paper_2511_16576_gb300 import evaluate as ev
    from paper_2511_16576_gb300 import synth
    dev = torch.device("cuda", ctx.device)
    n_train = min(args.train_queries, 8000)
    tq = synth.perturbed_queries(db, n_train, w.query_seed + 2000)
    tp = B.poly_upload(ctx, torch.from_numpy(tq.xy).to(dev), torch.from_numpy(tq.offsets).to(dev))
    s = ev.Searcher(ctx, index, P, dbp, h, shortlist=args.shortlist)
    feat, lab = ev.training_pairs(ctx, s, tp)
    rr = B.Reranker(ctx, seed=1)
    losses, secs = ev.timed(lambda: ev.train_reranker(rr, feat, lab, epochs=8))
    tp.close()
    return rr, {"pairs": int(feat.shape[0]), "loss_per_epoch": losses, "seconds": secs}


def main():
    args = parse()
    from paper_2511_16576_gb300 import synth
    w = synth.WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, w)
        return
    if args.paper_sweep:
        paper_sweep(args)
        return
    assert args.warmup >= 3 or os.environ.get("PMH_BENCH_ALLOW_SHORT"), "warm-up >= 3"

    import torch
    import torch.distributed as dist

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_2511_16576_gb300 import binding as B
    from paper_2511_16576_gb300 import build as cuda_build
    from paper_2511_16576_gb300 import dist as D
    from paper_2511_16576_gb300 import evaluate as ev
    cuda_build.build()

    dev = torch.device("cuda", local)
    # every rank signs and indexes its own shard of the same size (weak scaling)
    gen_w = D.shard_workload(w, rank)
    t_gen = time.perf_counter()
    db = synth.make_database(gen_w, args.n_polys)
    qs = synth.make_queries(gen_w, db, args.n_queries)
    t_gen = time.perf_counter() - t_gen
    N, Q, K = db.n, qs.n, w.K
    P = B.make_params(K, w.bands, w.T, w.seed, w.lsh_seed,
                      0 if args.no_stream_index else B.FLAG_STREAM_INDEX)
    ctx = B.Context(local)
    stream = torch.cuda.current_stream()

    # the stream index (once per seed and K), timed on its own
    sidx_ms = None
    if not args.no_stream_index:
        _, t = ev.timed(lambda: B.stream_index_build(ctx, P))
        sidx_ms = t * 1e3

    autotune = None
    if not args.no_autotune:
        # the walk kernel's shape, picked on a 0.2 % sample of the workload (cached per GPU/K)
        sample = db.subset(np.linspace(0, db.n - 1, max(1, min(db.n, 20000)), dtype=np.int64))
        sp = B.poly_upload(ctx, torch.from_numpy(sample.xy).to(dev),
                           torch.from_numpy(sample.offsets).to(dev))
        best, ms = B.sign_autotune(ctx, sp, P, cache_key=f"{w.name}:{N}:flags{P.flags}")
        autotune = {"variant": best, "points_per_lane_x_warps": B.sign_variant_info(best),
                    "sample_ms": [round(t, 3) for t in ms]}
        sp.close()

    d_xy = torch.from_numpy(db.xy).to(dev)
    d_off = torch.from_numpy(db.offsets).to(dev)
    q_xy = torch.from_numpy(qs.xy).to(dev)
    # the library's polygon set, signatures and bucket index: built once, then reloaded
    # and rebuilt in place by every step (the query graph is captured on them)
    dbp = B.poly_upload(ctx, d_xy, d_off)
    h = B.minhash_sign(ctx, dbp, P)
    index = B.lsh_build(ctx, h, P)
    qp_all = B.poly_upload(ctx, q_xy, torch.from_numpy(qs.offsets).to(dev))
    cap = ev.batch_capacity(ctx, index, P, qp_all, args.batch)
    qp_all.close()
    rr, train = (None, None) if args.plain else train_for_step(args, w, B, ctx, db, dbp, h, index, P)
    batches = ev.make_batches(q_xy, qs.offsets, args.batch)
    # with several ranks every rank searches the query batches of all ranks (gathered) on its
    # own shard, so its graph holds world x the batch
    shard_base = int(D.shard_offsets(N, dev)[rank]) if world > 1 else 0
    kk = args.refine_k
    g = B.QueryGraph(ctx, index, world * args.batch, world * batches.max_vertices, world * cap,
                     args.topm, db=dbp, k=kk, rerank=rr, shortlist=args.shortlist)
    assert world == 1 or kk > 0, "the exchange merges refined top-k lists"

    def local_search(allq, k):
        g.run(allq.xy, allq.offsets)
        n = allq.n
        return g.ref_ids[:n].to(torch.int64), g.ref_j[:n]

    def query_pass(src, out_ids, out_j):
        """Every query batch through the graph (one rank), or through the exchange."""
        if world == 1:
            ev.run_batches(g, src, out_ids, out_j)
            return
        q0 = 0
        for xy, off, n in zip(src.xy, src.off, src.n):
            xy, off = xy.to(dev, non_blocking=True), off.to(dev, non_blocking=True)
            gid, gj = D.global_search(local_search, D.QueryBatch(None, xy, off), shard_base, kk)
            out_ids[q0:q0 + n].copy_(gid, non_blocking=True)
            out_j[q0:q0 + n].copy_(gj, non_blocking=True)
            q0 += n
    res_cols = kk if kk > 0 else args.topm   # refined top-k, else the top-m lists
    res_ids = torch.empty((Q, res_cols), dtype=torch.int32, device=dev)
    res_j = torch.empty((Q, res_cols), dtype=torch.float64, device=dev) if kk > 0 else None
    ev_sign = []

    def step(host: bool, record: bool):
        if host:
            B.poly_reload(dbp, h_xy, h_off)
        else:
            B.poly_reload(dbp, d_xy, d_off)
        if record:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B.sign_timing(ctx, True)   # per-kernel events inside the call, no host sync
        B.minhash_sign(ctx, dbp, P, out=h)
        if record:
            B.sign_timing(ctx, False)
            e1.record(stream)
            ev_sign.append((e0, e1))
        B.lsh_rebuild(ctx, index, h)
        if host:
            query_pass(hbatches, hres_ids, hres_j)
        else:
            query_pass(batches, res_ids, res_j)

    h_xy = h_off = hbatches = hres_ids = hres_j = None
    if not args.no_e2e:
        h_xy = torch.from_numpy(db.xy).pin_memory()
        h_off = torch.from_numpy(db.offsets).pin_memory()
        hbatches = ev.make_batches(torch.from_numpy(qs.xy).pin_memory(), qs.offsets, args.batch,
                                   pinned=True)
        hres_ids = torch.empty((Q, res_cols), dtype=torch.int32).pin_memory()
        hres_j = torch.empty((Q, res_cols), dtype=torch.float64).pin_memory() if kk > 0 else None

    def timed(host: bool, steps: int, warmup: int, record: bool):
        for _ in range(warmup):
            step(host, False)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ev_sign.clear()
        l0 = B.launch_count()
        # (for a launch list under ncu: skip this many launches, capture one step's worth)
        print(json.dumps({"launches_before_timed": int(l0), "host_inputs": host}), file=sys.stderr,
              flush=True)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        profiled = args.cuda_profiler_range and not host
        if profiled:
            torch.cuda.profiler.start()
        t0.record(stream)
        for _ in range(steps):
            step(host, record)
        t1.record(stream)
        torch.cuda.synchronize()
        if profiled:
            torch.cuda.profiler.stop()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        launches = B.launch_count() - l0
        ms = D.max_over_ranks(t0.elapsed_time(t1) / steps, dev)
        return ms, launches

    clocks = Clocks(local)
    clocks.start()
    B.sign_report(ctx)                     # forget events of earlier calls
    B.sign_count_work(ctx, False)          # timed launches: the kernels without work counters
    ms, launches = timed(False, args.steps, args.warmup, True)
    clk = clocks.stop()
    flags = g.status()[0]
    sign_ms = float(np.mean([a.elapsed_time(b) for a, b in ev_sign]))
    kernel_ms = B.sign_report(ctx)         # mean per-kernel times of the timed database launches
    found = float((res_ids[:, 0] >= 0).float().mean())
    e2e = None
    if not args.no_e2e:
        ms_e2e, _ = timed(True, args.steps, args.warmup, False)
        h2d = db.xy.nbytes + db.offsets.nbytes + qs.xy.nbytes + 8 * (Q + len(batches.n))
        d2h = hres_ids.numel() * 4 + (hres_j.numel() * 8 if hres_j is not None else 0)
        e2e = {"value": world * (N + Q) * K / (ms_e2e * 1e-3), "unit": "hashes/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": ms_e2e}
        same = torch.equal(hres_ids, res_ids.cpu())
        e2e["results_equal_device_run"] = bool(same)

    # roofline of the dominant kernel: its algorithmic integer ops (work units it reports,
    # weighted as above) per launch / its mean CUDA-event time over the timed database
    # launches, against the measured integer peak; L2 / DRAM traffic from the ncu summary
    hashes_np = h.cpu().numpy().view(np.uint32)
    G = algorithmic_points(hashes_np, w.T)
    B.sign_count_work(ctx, True)
    B.minhash_sign(ctx, dbp, P, out=h)     # one more database launch, untimed, to read its work
    per_kernel = B.sign_report(ctx)        # work counts are fixed by the input: same as timed
    peak = B.probe_int_peak(ctx)
    kernels = {}
    for name, kname in (("unified", "sign_unified_kernel"), ("walk", "sign_kernel")):
        units = per_kernel[name]["work"]
        ops = sum(SIGN_OP_WEIGHTS[k] * v for k, v in units.items())
        kms = kernel_ms[name]["ms"]
        if kms <= 0.01 and ops == 0:
            continue
        kernels[kname] = {"ms": kms, "work_units_per_launch": units, "int_ops_per_launch": ops,
                          "achieved": ops / (kms * 1e-3) / 1e12 if kms > 0 else None,
                          "frac": ops / (kms * 1e-3) / peak if kms > 0 else None}
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    units = kernels[dom]["work_units_per_launch"]
    gather_bytes = 8 * (units["cells"] + units["index_entries"])
    prof = profiled_counters(N, w.name) if dom == "sign_unified_kernel" else None
    roofline = {"bound": "alu", "kernel": dom, "achieved": kernels[dom]["achieved"],
                "peak": peak / 1e12, "unit": "Tintop/s", "frac": kernels[dom]["frac"],
                "traffic": prof["dram_bytes"] if prof else None,
                "traffic_note": (f"ncu dram__bytes_read.sum + dram__bytes_write.sum of the same kernel "
                                 f"source on {prof['captured_on']}, x {prof['scale']:.2f} by polygons "
                                 f"({SIGN_PROFILE})") if prof else
                "no ncu summary of this kernel source on this workload: not measured",
                "op_weights": SIGN_OP_WEIGHTS,
                "peak_source": "measured: pmh_probe_int_peak (integer mad/add/xor/shl mix, all SMs)",
                "peak_nominal": nominal_int_peak(dev, clk),
                "kernels": kernels, "timed_launches": kernel_ms["calls"],
                # the index gather: cell records and entries read (8 B each), against the L2
                # sector bytes ncu counted for the launch
                "l2_gather": {"algorithmic_bytes": gather_bytes,
                              "lts_bytes": prof["lts_bytes"] if prof else None,
                              "lts_over_algorithmic": prof["lts_bytes"] / gather_bytes
                              if prof and gather_bytes else None,
                              "l2_throughput_pct_of_peak": prof["l2_throughput_pct"] if prof else None},
                "dram_throughput_pct_of_peak": prof["dram_throughput_pct"] if prof else None,
                "warp_inst_per_hash": prof["inst_executed"] / (N * K) if prof else None,
                "edge_tests_per_s": units["edge_tests"] / (kernels[dom]["ms"] * 1e-3),
                # the vertex stream (8 B per vertex, staged once per polygon by the signing
                # kernel) against the measured HBM copy bandwidth: far from being the bound
                "vertex_stream_gbs": db.xy.nbytes / (sign_ms * 1e-3) / 1e9,
                "vertex_stream_frac_of_hbm": db.xy.nbytes / (sign_ms * 1e-3) / 1e9 / hbm_peak_gbs()
                if hbm_peak_gbs() else None,
                "sign_ms": sign_ms, "stream_points_resolved": G,
                "stream_points_resolved_per_s": G / (sign_ms * 1e-3)}

    print(json.dumps({"timed_ms_per_step": ms, "sign_ms": sign_ms, "e2e": e2e, "launches": launches,
                      "launches_per_step": launches / args.steps,
                      "graph_status_flags": flags, "queries_with_a_result": found,
                      "unified_kernel_ms": kernels.get("sign_unified_kernel", {}).get("ms")}),
          file=sys.stderr, flush=True)
    batch_sizes = None
    if world == 1:
        # graph replays per batch size (1 .. 4,096 uneven queries) beside the same steps as
        # plain calls, both ranking by agreement count
        batch_sizes = ev.batch_size_sweep(ctx, index, P, dbp, h, q_xy, qs.offsets, m=args.topm,
                                          k=kk)
    search = None
    if not args.no_search and world == 1:
        search = search_quality(args, w, B, ctx, db, qs, h, dbp, q_xy,
                                torch.from_numpy(qs.offsets).to(dev), P)

    base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base = cpu_baseline(w, db, n_sample=args.cpu_sample)

    value = world * (N + Q) * K / (ms * 1e-3)
    line = {
        "metric": "polygon-hashes/s (N*K/s)", "value": value, "unit": "hashes/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": arm_config(args, w, db, Q, world),
        "sign_hashes_per_s": world * N * K / (sign_ms * 1e-3),
        "stream_index_build_ms": sidx_ms,
        "queries_per_s_in_step": world * Q / (ms * 1e-3),
        "query_batches_per_step": len(batches.n),
        "graph_status_flags": flags,
        "queries_with_a_result": found,
        "reranker_training": train,
        "roofline": roofline,
        "cpu_baseline": base,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "autotune": autotune,
        "graph_batch_sizes": batch_sizes,
        "search": search,
        "generation_seconds": t_gen,
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    g.close()
    if rr is not None:
        rr.close()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
