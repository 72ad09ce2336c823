"""Benchmark: batched HNSW search QPS at recall@10 >= 0.95 on 1M vectors.

Workload (the Sift1M-shaped case: 1,000,000 x 128, L2): base vectors are
integers 0..255 from a seeded 256-cluster mixture, 10,000 queries from the
same mixture, HNSW with M=32, efConstruction=200 built once on the host
(untimed).  A step is one batched search of the 10,000 queries: FP16
traversal (FP32 accumulation) followed by an exact FP32 re-rank of the
final ef candidates, at the smallest ef of the sweep 16..512 whose
recall@10 (against exact k-NN computed on the GPU) is >= 0.95.  The plain
FP32 traversal at the same ef is measured beside it.

`--impl reference` times the FP64 CPU oracle (the plain reference this
library is checked against) on a bounded sample of the same queries on the
same graph, on the host cores.

Multi-GPU (torchrun): every rank holds a full replica of the index and
searches its own 10,000 queries (no data-path collective; weak scaling).
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QPS at recall@10>=0.95, 1M vectors, 1 B300; FP16/PQ vs FP32; p99 ms"
N_BASE, N_QUERY, DIM, M, EFC, SEED, K = 1_000_000, 10_000, 128, 32, 200, 2, 10
EF_SWEEP = [16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512]
WORKLOAD = ("1M x 128 integer mixture (256 clusters, values 0..255), 10k queries, L2, HNSW M=32 efC=200, "
            "FP16 traversal + FP32 re-rank of ef, k=10")


def rank_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def shard_queries(rank, world, nq=N_QUERY, seed=SEED):
    """Queries of rank `rank` in a `world`-rank run (weak scaling): slice `rank`
    of one draw of world * nq queries, so the shards are disjoint; one rank gets
    the headline query set."""
    if world == 1:
        return make_workload(nq=nq, seed=seed)[1]
    return make_workload(n=1, nq=nq * world, seed=seed)[1][rank * nq:(rank + 1) * nq]


def max_over_ranks(x, world, device=None):
    """The largest of every rank's x (the job's time is its slowest rank's)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_qps(world, nq, steps, max_ms):
    """Whole-job throughput: the queries all ranks processed over the slowest
    rank's time."""
    return world * nq * steps / (max_ms / 1e3)


def make_workload(n=N_BASE, nq=N_QUERY, seed=SEED):
    from paper_2501_06121_b300 import datagen as G
    return G.integer_mixture(n, nq, d=DIM, clusters=256, sigma=20.0, seed=seed)


def graph_for(X, n, seed):
    """Host HNSW build (untimed input preparation), cached on local disk so
    that both benchmark arms on one machine share one graph."""
    from paper_2501_06121_b300 import kann as K_
    key = hashlib.sha1(("%d-%d-%d-%d-%d" % (n, DIM, M, EFC, seed)).encode()).hexdigest()[:12]
    path = os.path.join(tempfile.gettempdir(), "kann_bench_graph_%s.npz" % key)
    if os.path.exists(path):
        z = np.load(path)
        return {k: (z[k] if z[k].ndim else int(z[k])) for k in z.files}, 0.0, True
    t = time.time()
    g = K_.kann_hnsw_build_dense(X, K_.KANN_L2, M, EFC, seed, nthreads=0)
    dt = time.time() - t
    tmp = path + ".%d.tmp.npz" % os.getpid()
    np.savez(tmp, **g)
    os.replace(tmp, path)
    return g, dt, False


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, gpu):
        self.path = os.path.join(tempfile.gettempdir(), "kann_clocks_%d.csv" % os.getpid())
        q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu), "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                       "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self, t0, t1):
        """Summarise the samples taken between wall-clock times t0 and t1."""
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.p.terminate()
        self.p.wait()
        self.f.close()
        import datetime
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [s.strip() for s in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                if ts < t0 - 0.05 or ts > t1 + 0.05:
                    continue
                sm.append(float(parts[2]))
                mx.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[6:10]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.remove(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def recall_at(ids, gt, k=K):
    ids = ids[:, :k]
    gt = gt[:, :k]
    hit = (ids[:, :, None] == gt[:, None, :]).any(-1).sum(1)
    return float(hit.mean() / k)


class OracleRunner:
    """The FP64 oracle on this workload: FP16 traversal values with FP64
    arithmetic, then an FP64 re-rank on the FP32 vectors (the same path the
    GPU step runs), over a sample of the queries on all host cores."""

    def __init__(self, g, X, ef, threads=0, og=None):
        import oracle as O
        self.O = O
        self.og = og if og is not None else O.import_graph(g)
        self.Xh = O.encode_f16(X)
        self.X = X
        self.ef = ef
        self.threads = threads or (os.cpu_count() or 1)

    def run(self, Qs):
        O = self.O
        t = time.time()
        ti, _, cnt = O.search_dense(self.og, self.Xh, Qs, self.ef, self.ef, O.L2, dtype=O.DT_F16,
                                    nthreads=self.threads)
        O.rerank_dense(self.X, Qs, ti, K, O.L2)
        return time.time() - t

    def per_query_s(self, Q):
        n0 = min(len(Q), 8 * self.threads)
        return self.run(Q[:n0]) / n0

    def describe(self, n, total, dt):
        return {"value": n / dt, "unit": "queries/s", "cores": self.threads, "kind": "oracle",
                "sample": "%d queries of the %d-query set at ef=%d (FP16 traversal values, FP64 arithmetic, "
                          "FP64 re-rank), %.1f s on %d threads" % (n, total, self.ef, dt, self.threads)}


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_oracle_qps(g, X, Q, ef, seconds=12.0, sweep=(), point_seconds=0.8):
    """The FP64 oracle on the host: all cores at the selected ef (the line's
    value), one thread at the same ef (the paper's single-threaded query
    protocol, Sec. 3), and both over the ef sweep on bounded samples."""
    r = OracleRunner(g, X, ef)
    n = int(min(len(Q), max(8 * r.threads, seconds / max(r.per_query_s(Q), 1e-6))))
    dt = r.run(Q[:n])
    out = r.describe(n, len(Q), dt)
    out["cpu_model"] = cpu_model()
    r1 = OracleRunner(g, X, ef, threads=1, og=r.og)
    n1 = int(min(len(Q), max(4, 0.5 * seconds / max(r1.per_query_s(Q), 1e-6))))
    out["one_thread"] = {"value": n1 / r1.run(Q[:n1]), "unit": "queries/s", "cores": 1, "queries": n1}
    pts = []
    for e in sweep:
        p = {"ef": e}
        for name, runner in (("all_cores", r), ("one_thread", r1)):
            runner.ef = e
            per = runner.per_query_s(Q)
            m = int(min(len(Q), max(runner.threads, point_seconds / max(per, 1e-6))))
            p[name] = m / runner.run(Q[:m])
        pts.append(p)
    r.ef = r1.ef = ef
    out["by_ef"] = pts
    return out


def launch_kwargs(opts, work_ctr):
    """kann_search_ex keyword arguments for an autotuned option dict (the
    persistent form takes the preallocated work counter)."""
    o = dict(opts)
    if o.pop("persistent", False):
        o["work_counter"] = work_ctr
    return o


def select_ef(recalls, key, fixed=None):
    """The headline ef: the smallest of EF_SWEEP whose recall@10 (recalls(ef)[key])
    reaches 0.95, refined in quarter steps between the last sweep value below the
    target and it.  Returns (ef, {ef: recalls(ef)} for every ef tried)."""
    sweep = {}
    if fixed:
        sweep[fixed] = recalls(fixed)
        return fixed, sweep
    ef_sel = None
    for ef in EF_SWEEP:
        sweep[ef] = recalls(ef)
        if sweep[ef][key] >= 0.95:
            ef_sel = ef
            break
    if ef_sel is None:
        return EF_SWEEP[-1], sweep
    if ef_sel != EF_SWEEP[0]:
        lo = EF_SWEEP[EF_SWEEP.index(ef_sel) - 1]
        step = max(1, (ef_sel - lo) // 4)
        for efr in range(lo + step, ef_sel, step):
            sweep[efr] = recalls(efr)
            if sweep[efr][key] >= 0.95:
                ef_sel = efr
                break
    return ef_sel, sweep


def exact_ground_truth_cpu(X, Q, chunk=256):
    """Top-K ids by (distance, id) on the host.  On this workload (integers
    0..255, d = 128) every norm and dot product is an integer below 2^24, so the
    FP32 matmul and xn + qn - 2 q.x are exact; ties go to the lower id through the
    key distance * 2^20 + id (exact in FP64 for n <= 2^20)."""
    import torch
    Xt = torch.from_numpy(X)
    xn = (Xt.double() ** 2).sum(1)
    ids_col = torch.arange(X.shape[0], dtype=torch.float64)
    out = np.empty((len(Q), K), np.int64)
    for b in range(0, len(Q), chunk):
        Qt = torch.from_numpy(Q[b:b + chunk])
        dot = (Qt @ Xt.T).double()
        dist = xn[None, :] + (Qt.double() ** 2).sum(1)[:, None] - 2.0 * dot
        key = dist * float(1 << 20) + ids_col[None, :]
        out[b:b + chunk] = torch.topk(key, K, dim=1, largest=False, sorted=True).indices.numpy()
    return out


def run_reference(args):
    r, world, _ = rank_info()
    if r != 0:
        return
    X, Q = make_workload()
    g, _, _ = graph_for(X, N_BASE, SEED)
    runner = OracleRunner(g, X, args.ef or 64)
    if args.ef:
        ef = args.ef
    else:
        # the same ef rule as the GPU arm, with recall from the oracle's own
        # search; on this integer data the GPU search equals the oracle bit for
        # bit, so on the same graph both arms arrive at the same ef
        gt_cpu = exact_ground_truth_cpu(X, Q)

        def oracle_recalls(e):
            ti, _, _ = runner.O.search_dense(runner.og, runner.Xh, Q, e, e, runner.O.L2, dtype=runner.O.DT_F16,
                                             nthreads=runner.threads)
            oi, _ = runner.O.rerank_dense(X, Q, ti, K, runner.O.L2)
            return {"recall": recall_at(oi, gt_cpu)}

        ef, _ = select_ef(oracle_recalls, "recall")
    runner.ef = ef
    budget = max(0.2, 150.0 / max(1, args.steps + args.warmup))
    n_step = int(max(runner.threads, min(len(Q), budget / max(runner.per_query_s(Q), 1e-6))))
    pos = 0

    def step():
        nonlocal pos
        idx = (np.arange(n_step) + pos) % len(Q)
        pos = (pos + n_step) % len(Q)
        return runner.run(Q[idx])

    for _ in range(args.warmup):
        step()
    total_t = sum(step() for _ in range(args.steps))
    total_q = n_step * args.steps
    v = total_q / total_t
    base = runner.describe(total_q, len(Q), total_t)
    base["sample"] += "; %d queries per step" % n_step
    base["cpu_model"] = cpu_model()
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "queries/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * total_t / max(1, args.steps), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "ef": ef, "k": K, "queries_per_step": n_step},
           "cpu_baseline": base, "e2e": {"value": v, "unit": "queries/s", "h2d_bytes_per_step": 0,
                                         "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_serving(dev, args):
    """Continuous-batching serving of two resident indices: the 10k x 128
    Gaussian mixture (32 clusters, sigma 5; M=16, efC=100) and a 768-d index
    (`--serving-768-n` unit vectors, inner product, the concentrated mixture
    normalize(mu + 0.04 g) over 1,024 directions, M=32, efC=200, graph built
    on the device), both with FP8 E4M3 per-vector-scaled traversal and an FP32
    re-rank of the ef candidates (`--serving-pq`: the 768-d index also served
    with PQ m=192 codes, uint8 table, re-rank of 100, as a second run).
    Poisson arrivals at each rate for `--serving-seconds`, k in {10, 100},
    ef uniform in 64..512; latency = completion seen on the host - arrival.
    Admission by device memory (pages created and released within
    `--serving-memory` bytes).  For each index the served form's recall@10 and
    the plain FP32 traversal's at ef 128, the difference, and the largest
    relative error of the served distances against the FP64 oracle's
    distances of the same ids, on a sample of queries."""
    import oracle as O
    import torch
    from paper_2501_06121_b300 import datagen as G
    from paper_2501_06121_b300 import kann as K_
    from paper_2501_06121_b300 import serving as S
    X1, Q1 = G.gaussian_mixture(10000, 1000, d=128, clusters=32, sigma=5.0, seed=1)
    g1 = K_.kann_hnsw_build_dense(X1, K_.KANN_L2, 16, 100, 1, nthreads=0)
    X1d = torch_from(X1, dev)
    c1, s1 = K_.kann_quantize(X1d, K_.KANN_E4M3)
    small = K_.kann_index_upload(K_.graph_to_device(g1, dev), vectors=c1, dtype=K_.KANN_E4M3, scale=s1,
                                 metric=K_.KANN_L2, rerank=X1d)
    n7 = args.serving_768_n
    t0 = time.time()
    X7, Q7 = G.vmf_mixture(n7, 10_000, d=768, clusters=1024, kappa=50.0, seed=3, concentration=0.04)
    X7d = torch_from(X7, dev)
    del X7
    g7 = K_.kann_hnsw_build_device(X7d, K_.KANN_IP, 32, 200, 3)
    build7 = time.time() - t0
    gd7 = K_.graph_to_device(g7, dev)
    c7, s7 = K_.kann_quantize(X7d, K_.KANN_E4M3)
    big = K_.kann_index_upload(gd7, vectors=c7, dtype=K_.KANN_E4M3, scale=s7, metric=K_.KANN_IP, rerank=X7d)
    plain = {"10kx128": K_.kann_index_upload(K_.graph_to_device(g1, dev), vectors=X1d, metric=K_.KANN_L2),
             "768": K_.kann_index_upload(gd7, vectors=X7d, metric=K_.KANN_IP)}

    def accuracy(name, index, Xd_, Qh, metric, oracle_X, n=200, ef=128, opts=None):
        Qs = torch_from(Qh[:n], dev)
        gt, _ = K_.kann_exact_knn(Qs, Xd_, 10, metric)
        ids, d = K_.kann_search_ex(index, Qs, 10, ef, **(opts or dict(rerank=-1)))
        pi, _ = K_.kann_search_ex(plain[name], Qs, 10, ef)
        torch.cuda.synchronize()
        ids, d, gt, pi = ids.cpu().numpy(), d.cpu().numpy(), gt.cpu().numpy(), pi.cpu().numpy()
        ref = O.dist_dense(oracle_X, Qh[:n], np.maximum(ids, 0), metric)
        mag = np.abs(ref) if metric == K_.KANN_L2 else np.einsum(
            "qd,qkd->qk", np.abs(Qh[:n].astype(np.float64)), np.abs(oracle_X.astype(np.float64)[np.maximum(ids, 0)]))
        err = np.abs(d.astype(np.float64) - ref) / np.maximum(np.maximum(np.abs(ref), mag), 1e-30)
        r_s, r_p = recall_at(ids, gt), recall_at(pi, gt)
        return {"ef": ef, "queries": n, "recall@10_served": r_s, "recall@10_fp32_traversal": r_p,
                "recall_delta": r_s - r_p, "max_rel_dist_error_vs_fp64_oracle": float(err[ids >= 0].max())}

    acc = {"10kx128": accuracy("10kx128", small, X1d, Q1, K_.KANN_L2, X1),
           "768": accuracy("768", big, X7d, Q7, K_.KANN_IP, X7d.cpu().numpy())}
    # dense indices: `--serving-team` warps per query (0 = one warp)
    spec = dict(kmax=100, efmax=512, opts=dict(rerank=-1, team=args.serving_team))
    runs = [("e4m3_rerank", {"10kx128": dict(spec, index=small, d=128), "768": dict(spec, index=big, d=768)})]
    if args.serving_pq:
        cb = K_.kann_pq_train(X7d[:min(n7, 100_000)].contiguous(), 192, iters=25, seed=3)
        codes = K_.kann_pq_encode(X7d, cb)
        pq7 = K_.kann_index_upload(gd7, pq=dict(codes=codes, codebooks=cb, metric=K_.KANN_IP), rerank=X7d)
        acc["768_pq"] = accuracy("768", pq7, X7d, Q7, K_.KANN_IP, X7d.cpu().numpy(),
                                 opts=dict(rerank=100, pq_lut=K_.KANN_PQ_LUT_U8))
        runs.append(("pq_u8_rerank100", {"10kx128": dict(spec, index=small, d=128),
                                         "768": dict(kmax=100, efmax=512, index=pq7, d=768,
                                                     opts=dict(rerank=100, pq_lut=K_.KANN_PQ_LUT_U8))}))
    out = {"indices": {"10kx128": "10k x 128 Gaussian mixture, L2, M=16, efC=100",
                       "768": "%d x 768 unit vectors (concentrated mixture), IP, M=32, efC=200, device-built graph "
                              "(%.0f s incl. data)" % (n7, build7)},
           "traversal": "FP8 E4M3 per-vector scale + FP32 re-rank (R = ef)", "k": [10, 100], "ef": [64, 512],
           "seconds_per_rate": args.serving_seconds, "memory_budget": args.serving_memory,
           "team": args.serving_team,
           "accuracy_vs_fp64_oracle": acc, "runs": []}
    Q7h = Q7
    for run_name, indices in runs:
        tq = None if args.serving_no_tune else {"10kx128": torch_from(Q1[:500], dev), "768": torch_from(Q7h[:500], dev)}
        srv = S.SearchServer(indices, page_capacity=2048, memory_budget=args.serving_memory, max_pages=8,
                             tune_queries=tq)
        srv.prepare({"10kx128": 2, "768": 2})
        res = {"run": run_name, "page_capacity": srv.caps, "launch_settings_tuned": srv.tuned, "rates": []}
        for i, rate in enumerate(float(r) for r in args.serving_rates.split(",")):
            reqs = S.poisson_requests(rate, args.serving_seconds, {"10kx128": Q1, "768": Q7h}, seed=100 + i)
            done = srv.run(reqs, time_limit=args.serving_seconds * 3 + 10)
            summ = S.latency_summary(done, max(r["t_done"] for r in done) if done else 1.0)
            summ.update(offered_qps=rate, requests=len(reqs), status=S.status_counts(done))
            res["rates"].append(summ)
            print(json.dumps({"serving": run_name, **summ}), flush=True)
        res["memory"] = dict(srv.stats)
        out["runs"].append(res)
        del srv
    return out


def torch_from(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def run_pq768(args, n=None, concentration=None):
    """The MS MARCO-shaped workload: 1M x 768 unit-norm vMF mixture (1,024
    directions, kappa 50), 10k queries, inner product, HNSW M=32 efC=200 on
    the FP32 vectors, PQ m=192 x 256 trained on the GPU on a 100k sample;
    ADC traversal with an exact FP32 re-rank of the best 100, k = 10 and 100;
    the plain FP32 traversal beside it.  Ground truth: exact FP32 k-NN."""
    import torch
    from paper_2501_06121_b300 import build as lib_build
    from paper_2501_06121_b300 import datagen as G
    from paper_2501_06121_b300 import kann as K_
    lib_build.build()
    dev = torch.device("cuda", 0)
    n = n or args.pq_n
    concentration = concentration if concentration is not None else args.pq_concentration
    t0 = time.time()
    X, Q = G.vmf_mixture(n, 10_000, d=768, clusters=1024, kappa=50.0, seed=3,
                         concentration=concentration if concentration > 0 else None)
    gen_s = time.time() - t0
    key = "pq768-%d-%g" % (X.shape[0], concentration)
    path = os.path.join(tempfile.gettempdir(), "kann_bench_graph_%s.npz" % key)
    t0 = time.time()
    if os.path.exists(path):
        z = np.load(path)
        g = {k: (z[k] if z[k].ndim else int(z[k])) for k in z.files}
    else:
        g = K_.kann_hnsw_build_dense(X, K_.KANN_IP, 32, 200, 3, nthreads=0)
        np.savez(path + ".tmp.npz", **g)
        os.replace(path + ".tmp.npz", path)
    build_s = time.time() - t0
    Xd = torch.from_numpy(X).to(dev)
    Qd = torch.from_numpy(Q).to(dev)
    del X
    cb = K_.kann_pq_train(Xd[:min(n, 100_000)].contiguous(), 192, iters=25, seed=3)
    codes = K_.kann_pq_encode(Xd, cb)
    gd = K_.graph_to_device(g, dev)
    idx_pq = K_.kann_index_upload(gd, pq=dict(codes=codes, codebooks=cb, metric=K_.KANN_IP), rerank=Xd)
    idx32 = K_.kann_index_upload(gd, vectors=Xd, dtype=K_.KANN_F32, metric=K_.KANN_IP)
    t0 = time.time()
    gt100, _ = K_.kann_exact_knn(Qd, Xd, 100, K_.KANN_IP)
    torch.cuda.synchronize()
    gt_s = time.time() - t0
    gt100 = gt100.cpu().numpy()

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
        e0.record()
        for _ in range(reps):
            out = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, out

    rows = []
    for k in (10, 100):
        for ef in (32, 64, 128, 256, 512, 1024):
            if ef < k or (k > 10 and ef < 128):
                continue
            ms, (ids, _) = timed(lambda: K_.kann_search_ex(idx_pq, Qd, k, ef, rerank=100 if k <= 100 else -1))
            r = recall_at(ids.cpu().numpy(), gt100, k)
            ms16, (ids16, _) = timed(lambda: K_.kann_search_ex(idx_pq, Qd, k, ef, rerank=100 if k <= 100 else -1,
                                                               pq_lut=K_.KANN_PQ_LUT_F16))
            r16 = recall_at(ids16.cpu().numpy(), gt100, k)
            ms8, (ids8, _) = timed(lambda: K_.kann_search_ex(idx_pq, Qd, k, ef, rerank=100 if k <= 100 else -1,
                                                             pq_lut=K_.KANN_PQ_LUT_U8))
            r8 = recall_at(ids8.cpu().numpy(), gt100, k)
            # the uint8 table with every beam entry re-ranked (R = ef): the
            # recall a fixed R of 100 caps at k = 100
            mse, (idse, _) = timed(lambda: K_.kann_search_ex(idx_pq, Qd, k, ef, rerank=-1, pq_lut=K_.KANN_PQ_LUT_U8))
            re_ = recall_at(idse.cpu().numpy(), gt100, k)
            ms32, (ids32, _) = timed(lambda: K_.kann_search_ex(idx32, Qd, k, ef))
            r32 = recall_at(ids32.cpu().numpy(), gt100, k)
            rows.append({"k": k, "ef": ef, "pq_rerank100_qps": 1e4 / (ms / 1e3), "pq_rerank100_recall": r,
                         "pq_f16table_rerank100_qps": 1e4 / (ms16 / 1e3), "pq_f16table_rerank100_recall": r16,
                         "pq_u8table_rerank100_qps": 1e4 / (ms8 / 1e3), "pq_u8table_rerank100_recall": r8,
                         "pq_u8table_rerank_ef_qps": 1e4 / (mse / 1e3), "pq_u8table_rerank_ef_recall": re_,
                         "fp32_qps": 1e4 / (ms32 / 1e3), "fp32_recall": r32})
            print(json.dumps(rows[-1]), flush=True)
    out = {"workload": "pq768", "n": n, "concentration": concentration,
           "metric": "QPS and recall@k over ef, n x 768 IP, PQ m=192 + FP32 re-rank of 100 vs plain FP32",
           "data_gen_s": gen_s, "graph_build_s": build_s,
           "ground_truth_s": gt_s, "rows": rows}
    print(json.dumps(out))


def run_sparse(args, n_docs=None):
    """The Splade-shaped workload: `--sparse-n` documents (default 1M) over a
    30,522-term vocabulary (nnz ~ Poisson(120), Zipf(1.1) terms, lognormal
    weights), 10k queries (nnz ~ Poisson(40)), inner product, HNSW M=32
    efC=200 built with the layer-0 insertions on the GPU (`--sparse-host-build`:
    the host builder); QPS over all queries, recall@10 against the GPU sparse
    brute force on the first 1,000 queries, and the roofline of the search
    kernel on its algorithmic bytes."""
    import torch
    from paper_2501_06121_b300 import build as lib_build
    from paper_2501_06121_b300 import datagen as G
    from paper_2501_06121_b300 import kann as K_
    lib_build.build()
    dev = torch.device("cuda", 0)
    n_docs = n_docs or args.sparse_n
    t0 = time.time()
    base, qs = G.sparse_zipf(n_docs, 10_000, vocab=30522, lam_doc=120, lam_query=40, seed=4)
    gen_s = time.time() - t0
    td = lambda c: (torch.from_numpy(c[0]).to(dev), torch.from_numpy(c[1].view(np.int16)).to(dev),
                    torch.from_numpy(c[2]).to(dev))
    b_d, q_d = td(base), td(qs)
    t0 = time.time()
    if args.sparse_host_build:
        g = K_.kann_hnsw_build_sparse(base, 32, 200, 4, nthreads=0)
    else:
        g = K_.kann_hnsw_build_device_sparse(b_d[0], b_d[1], b_d[2], 30522, 32, 200, 4)
    build_s = time.time() - t0
    idx = K_.kann_index_upload(K_.graph_to_device(g, dev), sparse=dict(indptr=b_d[0], terms=b_d[1], weights=b_d[2],
                                                                        vocab=30522))
    ngt = 1000
    q_gt = td((qs[0][:ngt + 1], qs[1][:qs[0][ngt]], qs[2][:qs[0][ngt]]))
    t0 = time.time()
    gt, _ = K_.kann_exact_knn_sparse(b_d, q_gt, 30522, 10)
    torch.cuda.synchronize()
    gt_s = time.time() - t0
    gt = gt.cpu().numpy()
    # algorithmic bytes of an evaluated document: its (term, weight) pairs and
    # its two offsets; the evaluated documents are neighbours of expanded
    # nodes, so their mean size is taken weighted by in-degree on layer 0
    lens = np.diff(base[0]).astype(np.float64)
    indeg = np.bincount(g["l0"][g["l0"] >= 0].ravel(), minlength=n_docs).astype(np.float64)
    doc_bytes = float((indeg * (lens * 6 + 16)).sum() / max(indeg.sum(), 1.0))
    q_bytes = float(np.diff(qs[0]).mean() * 6 + 16)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6400.0)
    from paper_2501_06121_b300 import autotune as A_
    rows = []
    # the search sweep in an NVTX range named "search", so that a profiler
    # can take its launches apart from the graph build's
    torch.cuda.nvtx.range_push("search")
    for ef in (32, 64, 128, 256, 512, 1024):
        cnt = torch.zeros((len(qs[0]) - 1, 4), dtype=torch.int32, device=dev)
        K_.kann_search_sparse(idx, q_d[0], q_d[1], q_d[2], 10, ef, counters=cnt, hash_bits=15)
        torch.cuda.synchronize()
        c = cnt.double().mean(0).cpu().numpy()
        bq = c[0] * doc_bytes + c[1] * 64 * 4 + c[2] * doc_bytes + c[3] * 32 * 4 + q_bytes + 10 * 8
        # launch settings (visited table size, team size) by timing; every
        # one returns the same results, which is checked
        opts, ms, (ids, _) = fastest(lambda **o: K_.kann_search_sparse(idx, q_d[0], q_d[1], q_d[2], 10, ef, **o),
                                     [dict(hash_bits=hb, team=t) for hb in (12, 13, 14) for t in (0, 2, 4)])
        rows.append({"ef": ef, "qps": 1e4 / (ms / 1e3), "ms": ms,
                     "recall@10": recall_at(ids.cpu().numpy()[:ngt], gt, 10),
                     "docs_evaluated_per_query": c[0] + c[2], "algorithmic_bytes_per_query": bq,
                     "roofline_frac": 1e4 * bq / (ms / 1e3) / 1e9 / hbm, "launch": opts})
        print(json.dumps(rows[-1]), flush=True)
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"workload": "sparse", "docs": n_docs, "data_gen_s": gen_s, "graph_build_s": build_s,
                      "graph_builder": "host" if args.sparse_host_build else "device",
                      "doc_bytes_indegree_weighted": doc_bytes, "peak_gbs": hbm,
                      "ground_truth_s_1000q": gt_s, "rows": rows}))


def fastest(run, options, reps=3):
    """Times run(**o) for each option dict (CUDA events, after one untimed
    call) and returns (option, ms, output) of the fastest whose output equals
    the first option's bit for bit (launch settings never change results;
    one that did would be a fault, and is not chosen)."""
    import torch
    best = None
    ref = None
    for o in options:
        try:
            out = run(**o)
        except RuntimeError:
            continue
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
        e0.record()
        for _ in range(reps):
            out = run(**o)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        if ref is None:
            ref = out
        same = all(torch.equal(a, b) for a, b in zip(out, ref))
        if same and (best is None or ms < best[1]):
            best = (dict(o), ms, out)
    return best


def run_big(args):
    """The MS MARCO Star/Dragon-sized stand-in (Sec. 3, Table 1: 8,841,823
    passages, 768-d, inner product): `--big-n` unit vectors of the
    concentrated mixture normalize(mu + 0.04 g) over 1,024 directions,
    generated block by block straight to the device, 10k queries; HNSW M=32,
    efC=200 built with the layer-0 insertions on the GPU; PQ m=192 trained on
    the GPU on 100k rows, searched with the uint8 table and an FP32 re-rank of
    the best 100, beside plain FP32 traversal; ground truth: exact FP32 k-NN of
    the first 1,000 queries."""
    import torch
    from paper_2501_06121_b300 import build as lib_build
    from paper_2501_06121_b300 import datagen as G
    from paper_2501_06121_b300 import kann as K_
    lib_build.build()
    dev = torch.device("cuda", 0)
    n, d = args.big_n, 768
    t0 = time.time()
    blocks, Q = G.vmf_mixture_blocks(n, 10_000, d=d, clusters=1024, kappa=50.0, seed=3, concentration=0.04)
    Xd = torch.empty((n, d), dtype=torch.float32, device=dev)
    for s0, blk in blocks:
        Xd[s0:s0 + len(blk)].copy_(torch.from_numpy(blk))
    torch.cuda.synchronize()
    gen_s = time.time() - t0
    t0 = time.time()
    g = K_.kann_hnsw_build_device(Xd, K_.KANN_IP, 32, 200, 3)
    build_s = time.time() - t0
    t0 = time.time()
    cb = K_.kann_pq_train(Xd[:100_000].contiguous(), 192, iters=25, seed=3)
    codes = K_.kann_pq_encode(Xd, cb)
    torch.cuda.synchronize()
    pq_s = time.time() - t0
    gd = K_.graph_to_device(g, dev)
    del g
    Qd = torch.from_numpy(Q).to(dev)
    idx_pq = K_.kann_index_upload(gd, pq=dict(codes=codes, codebooks=cb, metric=K_.KANN_IP), rerank=Xd)
    idx32 = K_.kann_index_upload(gd, vectors=Xd, dtype=K_.KANN_F32, metric=K_.KANN_IP)
    # the BF16 re-rank copy (half the re-rank bytes; its distances are FP32
    # arithmetic on BF16-rounded rows)
    Xb, _ = K_.kann_quantize(Xd, K_.KANN_BF16)
    idx_pqb = K_.kann_index_upload(gd, pq=dict(codes=codes, codebooks=cb, metric=K_.KANN_IP), rerank=Xb)
    ngt = 1000
    t0 = time.time()
    gt, _ = K_.kann_exact_knn(Qd[:ngt].contiguous(), Xd, 10, K_.KANN_IP)
    torch.cuda.synchronize()
    gt_s = time.time() - t0
    gt = gt.cpu().numpy()

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
        e0.record()
        for _ in range(reps):
            out = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, out

    rows = []
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6400.0)

    def work(index, ef, **o):
        # mean per-query counters with a visited table that never forgets:
        # layer-0 evaluations, expansions, upper evaluations, upper hops
        cnt = torch.zeros((len(Q), 4), dtype=torch.int32, device=dev)
        K_.kann_search_ex(index, Qd, 10, ef, counters=cnt, hash_bits=15, visited_format=K_.KANN_VISITED_COMPACT, **o)
        torch.cuda.synchronize()
        return cnt.double().mean(0).cpu().numpy()

    torch.cuda.nvtx.range_push("search")  # the sweep, apart from the build (for a profiler)
    for ef in (16, 32, 48, 64, 128, 256, 512, 1024):
        # algorithmic bytes per query (row bytes x evaluations, adjacency rows,
        # the query, the output; PQ: 192-byte codes plus the re-rank rows)
        c32 = work(idx32, ef)
        b32 = (c32[0] + c32[2]) * d * 4 + c32[1] * 64 * 4 + c32[3] * 32 * 4 + d * 4 + 10 * 8
        c8 = work(idx_pq, ef, rerank=100, pq_lut=K_.KANN_PQ_LUT_U8)
        b8 = (c8[0] + c8[2]) * 192 + c8[1] * 64 * 4 + c8[3] * 32 * 4 + d * 4 + 10 * 8 + min(100, ef) * d * 4
        ms8, (i8, _) = timed(lambda: K_.kann_search_ex(idx_pq, Qd, 10, ef, rerank=100, pq_lut=K_.KANN_PQ_LUT_U8))
        msb, (ib, _) = timed(lambda: K_.kann_search_ex(idx_pqb, Qd, 10, ef, rerank=100, pq_lut=K_.KANN_PQ_LUT_U8))
        # re-rank of every beam entry (R = ef): lifts the cap a fixed R puts on recall
        mse, (ie, _) = timed(lambda: K_.kann_search_ex(idx_pq, Qd, 10, ef, rerank=-1, pq_lut=K_.KANN_PQ_LUT_U8))
        o32, ms32, (i32, _) = fastest(lambda **o: K_.kann_search_ex(idx32, Qd, 10, ef, **o),
                                      [dict(team=t, hash_bits=hb) for t in (0, 2, 4) for hb in (0, 13, 14)])
        rows.append({"ef": ef, "pq_u8table_rerank100_qps": 1e4 / (ms8 / 1e3),
                     "pq_u8table_rerank100_recall": recall_at(i8.cpu().numpy()[:ngt], gt),
                     "pq_u8table_bf16rerank100_qps": 1e4 / (msb / 1e3),
                     "pq_u8table_bf16rerank100_recall": recall_at(ib.cpu().numpy()[:ngt], gt),
                     "pq_u8table_rerank_ef_qps": 1e4 / (mse / 1e3),
                     "pq_u8table_rerank_ef_recall": recall_at(ie.cpu().numpy()[:ngt], gt),
                     "fp32_qps": 1e4 / (ms32 / 1e3), "fp32_recall": recall_at(i32.cpu().numpy()[:ngt], gt),
                     "fp32_launch": o32, "fp32_rows_evaluated_per_query": c32[0] + c32[2],
                     "fp32_algorithmic_bytes_per_query": b32,
                     "fp32_roofline_frac": 1e4 * b32 / (ms32 / 1e3) / 1e9 / hbm,
                     "pq_rows_evaluated_per_query": c8[0] + c8[2], "pq_u8_algorithmic_bytes_per_query": b8,
                     "pq_u8_roofline_frac": 1e4 * b8 / (ms8 / 1e3) / 1e9 / hbm})
        print(json.dumps(rows[-1]), flush=True)
    torch.cuda.nvtx.range_pop()
    dev_bytes = {"fp32_rows": n * d * 4, "bf16_rerank_rows": n * d * 2, "pq_codes": n * 192,
                 "graph_layer0": n * 64 * 4}
    print(json.dumps({"workload": "msmarco_dense", "n": n, "d": d, "data_gen_s": gen_s, "graph_build_s": build_s,
                      "graph_builder": "device", "pq_train_encode_s": pq_s, "ground_truth_s_1000q": gt_s,
                      "device_bytes": dev_bytes, "peak_gbs": hbm, "rows": rows}))


SEARCH_KERNEL_SOURCES = ("kann_device.cuh", "kann_internal.h", "kann_search_impl.cuh", "kann_search_f16.cu")


def search_kernel_sha():
    """SHA-1 over the sources of the FP16 dense search kernel, to tie stored
    DRAM counters to the kernel they were captured from."""
    h = hashlib.sha1()
    for name in SEARCH_KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2501_06121_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def traffic_from_profiles(kernel_sha, ef):
    """DRAM bytes (read + write) of one search launch at this ef, from the
    ncu counters stored in profiles/traffic.json, or None when none were taken
    for this kernel source and ef."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
        if t.get("kernel_source_sha1") == kernel_sha:
            return t.get("dram_bytes_per_launch_by_ef", {}).get(str(ef))
    except Exception:
        pass
    return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ef", type=int, default=0, help="fix ef instead of sweeping")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-curve", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="default launch settings instead of the autotuner's")
    ap.add_argument("--serving-seconds", type=float, default=8.0)
    ap.add_argument("--serving-768-n", type=int, default=1_000_000)
    ap.add_argument("--serving-pq", action="store_true", help="also serve the 768-d index with PQ codes")
    ap.add_argument("--serving-memory", type=int, default=48 << 20)
    ap.add_argument("--serving-team", type=int, default=0, help="warps per query of the dense served indices")
    ap.add_argument("--serving-no-tune", action="store_true", help="serve with default launch settings")
    ap.add_argument("--serving-rates", default="5000,20000,50000,100000,200000")
    ap.add_argument("--workload", default="sift1m",
                    choices=["sift1m", "pq768", "sparse", "sparse100k", "serving", "msmarco_dense"])
    ap.add_argument("--big-n", type=int, default=8_841_823)
    ap.add_argument("--sparse-n", type=int, default=1_000_000)
    ap.add_argument("--sparse-host-build", action="store_true")
    ap.add_argument("--pq-n", type=int, default=1_000_000)
    ap.add_argument("--pq-concentration", type=float, default=0.0,
                    help="> 0: normalize(mu + sigma g) mixture instead of the kappa=50 vMF draw")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "pq768":
        return run_pq768(args)
    if args.workload == "sparse100k":
        return run_sparse(args, n_docs=100_000)
    if args.workload == "sparse":
        return run_sparse(args)
    if args.workload == "msmarco_dense":
        return run_big(args)
    if args.workload == "serving":
        import torch
        from paper_2501_06121_b300 import build as lib_build
        lib_build.build()
        print(json.dumps({"workload": "serving", "serving": run_serving(torch.device("cuda", 0), args)}))
        return None

    import torch
    import torch.distributed as dist

    from paper_2501_06121_b300 import build as lib_build
    from paper_2501_06121_b300 import kann as K_

    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    lib_build.build()
    dev = torch.device("cuda", local)

    # ---- inputs (untimed)
    X, Q = make_workload(seed=SEED)
    if world > 1:
        Q = shard_queries(rank, world)
    t0 = time.time()
    if world > 1 and rank != 0:
        dist.barrier()
    g, build_s, cached = graph_for(X, N_BASE, SEED)
    if world > 1 and rank == 0:
        dist.barrier()
    Xd = torch.from_numpy(X).to(dev)
    Xh, _ = K_.kann_quantize(Xd, K_.KANN_F16)
    gd = K_.graph_to_device(g, dev)
    idx16 = K_.kann_index_upload(gd, vectors=Xh, dtype=K_.KANN_F16, metric=K_.KANN_L2, rerank=Xd)
    idx32 = K_.kann_index_upload(gd, vectors=Xd, dtype=K_.KANN_F32, metric=K_.KANN_L2)
    Qd = torch.from_numpy(Q).to(dev)
    # ground truth: tensor-core exact k-NN on BF16 copies (integers 0..255 are
    # exact in BF16 and every dot product / norm stays below 2^24 in FP32)
    Xb, _ = K_.kann_quantize(Xd, K_.KANN_BF16)
    Qb, _ = K_.kann_quantize(Qd, K_.KANN_BF16)
    torch.cuda.synchronize()
    tg = time.time()
    gt, gt_d = K_.kann_exact_knn(Qb, Xb, K, K_.KANN_L2, dtype=K_.KANN_BF16)
    torch.cuda.synchronize()
    gt_s = time.time() - tg
    del Xb
    gt = gt.cpu().numpy()
    gt_kth = gt_d[:, K - 1].cpu().numpy().astype(np.float64)
    # the ground truth above is the library's tensor-core kernel; the FP64
    # oracle's brute force recomputes a sample of it independently
    gt_check = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle as O_
        n_chk = 24
        t_c = time.time()
        oi, od = O_.exact_dense(X, Q[:n_chk], K, O_.L2)
        gt_check = {"queries": n_chk, "ids_equal": bool(np.array_equal(oi, gt[:n_chk])),
                    "dists_equal": bool(np.array_equal(od, gt_d[:n_chk].cpu().numpy().astype(np.float64))),
                    "oracle_s": time.time() - t_c,
                    "rule": "oracle.exact_dense (FP64 brute force, ties to the lower id) on the first queries"}

    # ---- ef sweep: smallest ef with recall@10 >= 0.95 (FP16 + re-rank)
    def gpu_recalls(ef):
        ids, _ = K_.kann_search_ex(idx16, Qd, K, ef, rerank=-1)
        torch.cuda.synchronize()
        rec = recall_at(ids.cpu().numpy(), gt)
        i32, _ = K_.kann_search_ex(idx32, Qd, K, ef)
        torch.cuda.synchronize()
        return {"recall_fp16_rerank": rec, "recall_fp32": recall_at(i32.cpu().numpy(), gt)}

    ef, sweep = select_ef(gpu_recalls, "recall_fp16_rerank", args.ef)

    # algorithmic work per query (large visited table: no repeated distances)
    cnt = torch.zeros((N_QUERY, 4), dtype=torch.int32, device=dev)
    K_.kann_search_ex(idx16, Qd, K, ef, rerank=-1, counters=cnt, hash_bits=14)
    torch.cuda.synchronize()
    c = cnt.double().mean(0).cpu().numpy()
    row16, row32 = DIM * 2, DIM * 4
    bytes_per_q = (c[0] * row16 + c[1] * 2 * M * 4 + c[2] * row16 + c[3] * M * 4 + ef * row32
                   + DIM * 4 + K * 8)

    stream = torch.cuda.current_stream()

    ids_buf = torch.empty((N_QUERY, K), dtype=torch.int32, device=dev)
    d_buf = torch.empty((N_QUERY, K), dtype=torch.float32, device=dev)

    # launch settings per arm from the autotuner (every candidate must return
    # the default launch's ids and distances bit for bit)
    from paper_2501_06121_b300 import autotune as A_
    work_ctr = torch.zeros(1, dtype=torch.int32, device=dev)
    t_tune = time.time()
    tuned16 = A_.tune(idx16, Qd, K, ef, rerank=-1, reps=3) if not args.no_tune else {}
    tuned32 = A_.tune(idx32, Qd, K, ef, rerank=0, reps=3) if not args.no_tune else {}
    tune_s = time.time() - t_tune
    kw16, kw32 = launch_kwargs(tuned16, work_ctr), launch_kwargs(tuned32, work_ctr)

    def timed(index, rr, steps, warm, kw, label):
        for _ in range(warm):
            K_.kann_search_ex(index, Qd, K, ef, ids=ids_buf, dists=d_buf, rerank=rr, **kw)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        # the timed launches in an NVTX range of their own (a profiler can
        # select exactly these)
        torch.cuda.nvtx.range_push(label)
        evs[0].record(stream)
        for i in range(steps):
            K_.kann_search_ex(index, Qd, K, ef, ids=ids_buf, dists=d_buf, rerank=rr, **kw)
            evs[i + 1].record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        per = [evs[i].elapsed_time(evs[i + 1]) for i in range(steps)]
        return sum(per), per

    clocks = Clocks(local)
    time.sleep(0.3)
    w0 = time.time()
    total_ms, per = timed(idx16, -1, args.steps, args.warmup, kw16, "timed_fp16")
    clk = clocks.stop(w0 + 1e-3 * 0, time.time())
    total_ms = max_over_ranks(total_ms, world, dev)
    fp32_ms, _ = timed(idx32, 0, max(3, args.steps // 2), 2, kw32, "timed_fp32")
    fp32_ms /= max(3, args.steps // 2)

    qps = job_qps(world, N_QUERY, args.steps, total_ms)
    ms_step = total_ms / args.steps
    per_launch_s = ms_step / 1e3
    achieved = N_QUERY * bytes_per_q / per_launch_s / 1e9
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6400.0)
    traffic = traffic_from_profiles(search_kernel_sha(), ef)

    # ---- end to end through the public API with host buffers
    Qpin = torch.from_numpy(Q).pin_memory()
    ids_h = torch.empty((N_QUERY, K), dtype=torch.int32).pin_memory()
    d_h = torch.empty((N_QUERY, K), dtype=torch.float32).pin_memory()

    # every step copies its queries in and its results out; the copies of
    # neighbouring steps overlap the search on two copy streams
    # (serving.HostBatchPipeline); the persistent form keeps its own counter
    from paper_2501_06121_b300 import serving as S_
    kw_pipe = dict(kw16)
    if "work_counter" in kw_pipe:
        kw_pipe["work_counter"] = torch.zeros(1, dtype=torch.int32, device=dev)
    pipe = S_.HostBatchPipeline(idx16, N_QUERY, Qd.shape[1], K, ef, device=dev, rerank=-1, **kw_pipe)

    for _ in range(args.warmup):
        pipe.submit(Qpin, ids_h, d_h)
    pipe.synchronize()
    if world > 1:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(pipe.first_stream())
    for _ in range(args.steps):
        pipe.submit(Qpin, ids_h, d_h)
    e1.record(pipe.last_stream())  # after the last step's results reached the host
    pipe.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    e2e_ms = max_over_ranks(e2e_ms, world, dev)
    e2e_qps = job_qps(world, N_QUERY, args.steps, e2e_ms)
    # the results the end-to-end steps brought back to the host
    final_recall = recall_at(ids_h.numpy(), gt)
    # tie-aware recall: a returned id counts when its exact distance is within
    # the k-th ground-truth distance (equal distances are common on integer data)
    fd = d_h.numpy().astype(np.float64)
    fi = ids_h.numpy()
    tie_recall = float(((fd <= gt_kth[:, None]) & (fi >= 0)).sum(1).mean() / K)

    # recall-QPS curve over the ef sweep (untimed by the step clock; CUDA events
    # per point), with the achieved fraction of the HBM peak on algorithmic bytes
    curve = []
    if rank == 0 and not args.no_curve:
        for efc in EF_SWEEP:
            cc = torch.zeros((N_QUERY, 4), dtype=torch.int32, device=dev)
            K_.kann_search_ex(idx16, Qd, K, efc, rerank=-1, counters=cc, hash_bits=14)
            torch.cuda.synchronize()
            m = cc.double().mean(0).cpu().numpy()
            bq = m[0] * row16 + m[1] * 2 * M * 4 + m[2] * row16 + m[3] * M * 4 + efc * row32 + DIM * 4 + K * 8
            point = {"ef": efc, "l0_dist_per_query": m[0]}
            for name, index, rr, rb in (("fp16_rerank", idx16, -1, bq),
                                        ("fp32", idx32, 0, bq + m[0] * (row32 - row16) + m[2] * (row32 - row16)
                                         - efc * row32)):
                opt_c = A_.tune(index, Qd, K, efc, rerank=rr, reps=2) if not args.no_tune else {}
                kwc = launch_kwargs(opt_c, work_ctr)
                for _ in range(2):
                    K_.kann_search_ex(index, Qd, K, efc, rerank=rr, **kwc)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
                e0.record()
                for _ in range(5):
                    cid_, _ = K_.kann_search_ex(index, Qd, K, efc, rerank=rr, **kwc)
                e1.record()
                torch.cuda.synchronize()
                msc = e0.elapsed_time(e1) / 5
                point[name] = {"recall@10": recall_at(cid_.cpu().numpy(), gt), "qps": N_QUERY / (msc / 1e3),
                               "ms": msc, "roofline_frac": N_QUERY * rb / (msc / 1e3) / 1e9 / hbm,
                               "launch": opt_c}
            curve.append(point)

    # the multi-expansion layer-0 step (kann_search_opts.expand = p): its own
    # smallest ef with recall@10 >= 0.95, timed like the headline form
    multi = []
    if rank == 0 and not args.no_curve:
        for p_exp in (2, 4):
            def multi_recalls(e, p_exp=p_exp):
                ids_m, _ = K_.kann_search_ex(idx16, Qd, K, e, rerank=-1, expand=p_exp)
                torch.cuda.synchronize()
                return {"recall": recall_at(ids_m.cpu().numpy(), gt)}

            ef_m, _ = select_ef(multi_recalls, "recall")
            kwm = dict(kw16, expand=p_exp)
            for _ in range(3):
                K_.kann_search_ex(idx16, Qd, K, ef_m, rerank=-1, **kwm)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
            e0.record()
            for _ in range(10):
                ids_m, _ = K_.kann_search_ex(idx16, Qd, K, ef_m, rerank=-1, **kwm)
            e1.record()
            torch.cuda.synchronize()
            ms_m = e0.elapsed_time(e1) / 10
            multi.append({"expand": p_exp, "ef": ef_m, "recall@10": recall_at(ids_m.cpu().numpy(), gt),
                          "qps": N_QUERY / (ms_m / 1e3), "ms": ms_m,
                          "vs_one_expansion_qps": N_QUERY / (ms_m / 1e3) / qps})

    # the same graph built with the layer-0 insertions on the GPU: build time
    # and the headline form's recall at the selected ef on it
    build_dev = None
    if rank == 0 and not args.no_curve:
        torch.cuda.synchronize()
        t_b = time.time()
        g_dev = K_.kann_hnsw_build_device(Xd, K_.KANN_L2, M, EFC, SEED)
        t_b = time.time() - t_b
        idx_dev = K_.kann_index_upload(K_.graph_to_device(g_dev, dev), vectors=Xh, dtype=K_.KANN_F16, metric=K_.KANN_L2,
                                       rerank=Xd)
        rec_dev = {}
        for e in sorted(set([ef] + [x for x in EF_SWEEP if x <= 128])):
            ids_g, _ = K_.kann_search_ex(idx_dev, Qd, K, e, rerank=-1)
            ids_h, _ = K_.kann_search_ex(idx16, Qd, K, e, rerank=-1)
            torch.cuda.synchronize()
            rec_dev[str(e)] = {"device_graph": recall_at(ids_g.cpu().numpy(), gt),
                               "host_graph": recall_at(ids_h.cpu().numpy(), gt)}
        build_dev = {"device_build_s": t_b, "host_build_s": build_s if not cached else None,
                     "host_build_cached": cached, "recall@10_fp16_rerank": rec_dev,
                     "rule": "kann_hnsw_build_device: upper-layer nodes on the host, level-0 nodes on the GPU in "
                             "batches of 1/32 of the graph; same M, efConstruction and levels"}
        del idx_dev, g_dev

    serving = None
    if rank == 0 and world == 1 and not args.no_serving:
        serving = run_serving(dev, args)

    cpu_base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_base = cpu_oracle_qps(g, X, Q, ef, sweep=EF_SWEEP if not args.no_curve else ())

    if rank == 0:
        per_sorted = sorted(per)
        out = {
            "metric": METRIC, "value": qps, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "ef": ef, "k": K, "recall@10": final_recall,
                       "recall@10_tie_aware": tie_recall,
                       "storage": "f16 traversal + f32 re-rank (R = ef)", "parallelism": "replicas%d" % world,
                       "l2": "inputs larger than L2 (f16 base 256 MB + f32 base 512 MB + graph 256 MB)",
                       "fp32_plain_qps": N_QUERY * world / (fp32_ms / 1e3), "fp32_plain_ms_per_step": fp32_ms,
                       "ef_sweep": {str(e): sweep[e] for e in sorted(sweep)}, "graph_build_s": build_s,
                       "graph_cached": cached,
                       "ground_truth_s": gt_s,
                       "ground_truth": "tensor-core exact k-NN on BF16 copies (exact on this integer data)",
                       "ground_truth_check": gt_check,
                       "batch_latency_ms": {"p50": per_sorted[len(per) // 2],
                                            "p99": per_sorted[min(len(per) - 1, int(0.99 * len(per)))]},
                       "work_per_query": {"l0_dist": c[0], "l0_expansions": c[1], "upper_dist": c[2],
                                          "upper_hops": c[3]},
                       "launch_settings": {"fp16_rerank": tuned16, "fp32": tuned32, "tune_s": tune_s,
                                           "rule": "autotuner: fastest of the result-preserving settings "
                                                   "(visited table layout and size, lanes per row, warps "
                                                   "per CTA, team size, lean, persistent), same ids and distances "
                                                   "as the default launch"},
                       "host_cores": os.cpu_count()},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                         "traffic": traffic, "algorithmic_bytes_per_query": bytes_per_q,
                         "kernel": "search_dense_kernel<f16> (one launch per step)",
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy)" if peaks else "fallback"},
            "e2e": {"value": e2e_qps, "unit": "queries/s", "h2d_bytes_per_step": int(Q.nbytes),
                    "d2h_bytes_per_step": int(ids_h.numel() * 4 + d_h.numel() * 4),
                    "copies": "every step: queries from pinned host memory in, ids and distances out; the copies of "
                              "neighbouring steps overlap the search on two copy streams (serving.HostBatchPipeline)"},
            "gpu_launches": args.steps,
            "clocks": clk,
            "cpu_baseline": cpu_base,
            "serving": serving,
            "recall_qps_curve": curve,
            "multi_expansion": multi,
            "graph_build_device": build_dev,
        }
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
