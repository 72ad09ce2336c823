"""Continuous-batching search server over resident indices.

Requests (index, query, k, ef) arrive over time.  The server runs them in
batches on *pages*: a page belongs to one index and holds a CUDA stream,
device and pinned host buffers for up to `capacity` queries (queries, per-query
k and ef, outputs, per-query status words) and a CUDA graph of one
persistent, work-stealing `kann_search_batch` launch that reads the batch size
from device memory, so one graph serves any batch up to the capacity.

Admission is by device memory: every page counts the bytes
`kann_search_workspace_bytes` gives for its capacity and settings, and the
pages alive at any time never exceed the memory budget.  When requests of an
index are waiting and no page of that index is idle, the server creates one if
the budget has room, else releases the least recently used idle page of
another index that has no requests waiting and takes its memory, else the
requests wait until a running batch finishes and frees its page.  So arriving requests are admitted as
memory (not a fixed partition of it) frees up, batches of different indices
overlap on the device on their own streams, and a burst on one index can use
the memory that idle indices are not using.  Every finished request carries
its status word (KANN_QSTAT_* bits); the run's summary counts them.

Every search step runs in the library's kernels; this module only stages
buffers, replays graphs and keeps time.
"""
import collections
import time

import numpy as np
import torch

from . import kann as K


class _Page:
    def __init__(self, name, spec, cap, device, opts):
        self.name, self.index, self.d = name, spec["index"], spec["d"]
        self.kmax, self.efmax, self.cap = spec["kmax"], spec["efmax"], cap
        self.stream = torch.cuda.Stream(device=device)
        f32, i32 = torch.float32, torch.int32
        self.q = torch.zeros((cap, self.d), dtype=f32, device=device)
        self.k = torch.ones(cap, dtype=i32, device=device)
        self.ef = torch.full((cap,), self.kmax, dtype=i32, device=device)
        self.n = torch.zeros(1, dtype=i32, device=device)
        self.counter = torch.zeros(1, dtype=i32, device=device)
        self.ids = torch.empty((cap, self.kmax), dtype=i32, device=device)
        self.dists = torch.empty((cap, self.kmax), dtype=f32, device=device)
        self.status = torch.zeros(cap, dtype=i32, device=device)
        self.h_q = torch.zeros((cap, self.d), dtype=f32).pin_memory()
        self.h_k = torch.ones(cap, dtype=i32).pin_memory()
        self.h_ef = torch.full((cap,), self.kmax, dtype=i32).pin_memory()
        self.h_n = torch.zeros(1, dtype=i32).pin_memory()
        self.h_ids = torch.empty((cap, self.kmax), dtype=i32).pin_memory()
        self.h_dists = torch.empty((cap, self.kmax), dtype=f32).pin_memory()
        self.h_status = torch.zeros(cap, dtype=i32).pin_memory()
        self.np_q, self.np_k, self.np_ef = self.h_q.numpy(), self.h_k.numpy(), self.h_ef.numpy()
        self.np_ids, self.np_dists, self.np_status = self.h_ids.numpy(), self.h_dists.numpy(), self.h_status.numpy()
        self.opts = opts
        self.event = torch.cuda.Event()
        self.busy = None  # the requests in flight
        self.last_used = 0.0
        self.bytes = K.kann_search_workspace_bytes(self.index, cap, self.kmax, self.efmax, **self._size_opts())
        self._capture()

    def _size_opts(self):
        return {k: v for k, v in self.opts.items() if k not in ("status", "counters", "work_counter", "n_device")}

    def _launch(self):
        K.kann_search_batch(self.index, self.q, self.k, self.ef, kmax=self.kmax, efmax=self.efmax, ids=self.ids,
                            dists=self.dists, stream=self.stream, work_counter=self.counter, n_device=self.n,
                            status=self.status, **self.opts)

    def _capture(self):
        # warm the launch once (sets kernel attributes), then capture it
        self.h_n[0] = 1
        with torch.cuda.stream(self.stream):
            self.n.copy_(self.h_n, non_blocking=True)
            self._launch()
        self.stream.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream, capture_error_mode="relaxed"):
            self._launch()
        self.stream.synchronize()

    def submit(self, reqs):
        n = len(reqs)
        self.np_q[:n] = np.stack([r["query"] for r in reqs])
        self.np_k[:n] = [r["k"] for r in reqs]
        self.np_ef[:n] = [r["ef"] for r in reqs]
        self.h_n[0] = n
        with torch.cuda.stream(self.stream):
            self.q[:n].copy_(self.h_q[:n], non_blocking=True)
            self.k[:n].copy_(self.h_k[:n], non_blocking=True)
            self.ef[:n].copy_(self.h_ef[:n], non_blocking=True)
            self.n.copy_(self.h_n, non_blocking=True)
            self.graph.replay()
            self.h_ids[:n].copy_(self.ids[:n], non_blocking=True)
            self.h_dists[:n].copy_(self.dists[:n], non_blocking=True)
            self.h_status[:n].copy_(self.status[:n], non_blocking=True)
            self.event.record(self.stream)
        self.busy = reqs

    def poll(self):
        """Finished requests (with results and status filled in), or None if
        still running."""
        if self.busy is None or not self.event.query():
            return None
        reqs, self.busy = self.busy, None
        for i, r in enumerate(reqs):
            r["ids"] = self.np_ids[i, :r["k"]].copy()
            r["dists"] = self.np_dists[i, :r["k"]].copy()
            r["status"] = int(self.np_status[i])
        return reqs


class SearchServer:
    """indices: {name: dict(index=Index, d=..., kmax=..., efmax=..., opts={...})}.

    page_capacity: queries per batch (halved for an index until one page fits
    the budget); memory_budget: device bytes all live pages may count
    together (each page counts kann_search_workspace_bytes of its capacity);
    max_pages: streams in flight at most.  tune_queries ({name: device
    [m, d] FP32 queries}, dense and PQ indices): the index's launch settings
    are chosen by the autotuner on those queries at k = min(10, kmax) and
    ef = efmax / 2 (result-preserving settings only; `tuned` records them)."""

    def __init__(self, indices, page_capacity=1024, memory_budget=1 << 30, max_pages=16, device="cuda",
                 search_opts=None, tune_queries=None):
        self.specs, self.caps, self.page_bytes, self.tuned = {}, {}, {}, {}
        self.device, self.budget, self.max_pages = device, memory_budget, max_pages
        for name, spec in indices.items():
            opts = dict(search_opts or {}, **spec.get("opts", {}))
            if tune_queries and name in tune_queries:
                from . import autotune
                k = min(10, spec["kmax"])
                got = autotune.tune(spec["index"], tune_queries[name], k, max(k, spec["efmax"] // 2),
                                    rerank=opts.get("rerank", 0), reps=3, fixed=opts)
                got.pop("persistent", None)
                self.tuned[name] = got
                opts.update({key: v for key, v in got.items() if v})
            opts.pop("persistent", None)  # pages always launch the persistent form
            size = lambda c: K.kann_search_workspace_bytes(spec["index"], c, spec["kmax"], spec["efmax"], **opts)
            cap = page_capacity
            if size(cap) == 0:
                raise ValueError("index %r cannot run a search with kmax=%d efmax=%d" % (name, spec["kmax"],
                                                                                        spec["efmax"]))
            while cap > 16 and size(cap) > memory_budget:
                cap //= 2
            if size(cap) > memory_budget:
                raise ValueError("index %r: a page of %d queries needs %d bytes, above the budget" %
                                 (name, cap, size(cap)))
            self.specs[name] = dict(spec, opts=opts)
            self.caps[name] = cap
            self.page_bytes[name] = size(cap)
        self.pages = []
        self.stats = {"pages_created": 0, "pages_released": 0, "admissions_waited_for_memory": 0,
                      "peak_bytes": 0}

    # ---- pages
    def live_bytes(self):
        return sum(p.bytes for p in self.pages)

    def _new_page(self, name):
        p = _Page(name, self.specs[name], self.caps[name], self.device, self.specs[name]["opts"])
        self.pages.append(p)
        self.stats["pages_created"] += 1
        self.stats["peak_bytes"] = max(self.stats["peak_bytes"], self.live_bytes())
        return p

    def _page_for(self, name, pending):
        """An idle page of index `name`, made room for within the budget, or
        None when the memory is taken by running batches and by pages of
        indices that have requests waiting."""
        for p in self.pages:
            if p.name == name and p.busy is None:
                return p
        need = self.page_bytes[name]
        if self.live_bytes() + need <= self.budget and len(self.pages) < self.max_pages:
            return self._new_page(name)
        # release idle pages of other indices that have nothing waiting (a
        # page of an index with waiting requests is about to be used again:
        # taking it would only trade captures); an index's last page goes
        # only after every spare one, least recently used first
        idle = [p for p in self.pages if p.busy is None and p.name != name and not pending[p.name]]
        while idle and not (self.live_bytes() + need <= self.budget and len(self.pages) < self.max_pages):
            held = collections.Counter(q.name for q in self.pages)
            p = min(idle, key=lambda q: (held[q.name] <= 1, q.last_used))
            idle.remove(p)
            self.pages.remove(p)
            self.stats["pages_released"] += 1
        if self.live_bytes() + need <= self.budget and len(self.pages) < self.max_pages:
            return self._new_page(name)
        return None

    def prepare(self, counts=None):
        """Create pages up front (counts: {name: pages}) so that the first
        requests do not pay for a graph capture."""
        for name, c in (counts or {n: 1 for n in self.specs}).items():
            for _ in range(c):
                if self.live_bytes() + self.page_bytes[name] > self.budget or len(self.pages) >= self.max_pages:
                    break
                self._new_page(name)

    # ---- serving
    def run(self, requests, time_limit=None):
        """requests: list of dict(t=arrival seconds from start, index=name,
        query=float32[d], k=int, ef=int).  Serves them in arrival order,
        sleeping until each arrives; returns them with 'ids', 'dists',
        'status', 't_done' (seconds from start) and 'latency' (t_done - t)."""
        reqs = sorted(requests, key=lambda r: r["t"])
        pending = {name: collections.deque() for name in self.specs}
        nxt, done = 0, []
        t0 = time.perf_counter()
        waited = set()
        while len(done) < len(reqs):
            now = time.perf_counter() - t0
            if time_limit is not None and now > time_limit:
                break
            while nxt < len(reqs) and reqs[nxt]["t"] <= now:
                pending[reqs[nxt]["index"]].append(reqs[nxt])
                nxt += 1
            for p in self.pages:
                fin = p.poll()
                if fin is not None:
                    tnow = time.perf_counter() - t0
                    p.last_used = tnow
                    for r in fin:
                        r["t_done"] = tnow
                        r["latency"] = tnow - r["t"]
                    done.extend(fin)
            # admit: the index whose oldest waiting request is oldest goes first
            order = sorted((q[0]["t"], name) for name, q in pending.items() if q)
            for _, name in order:
                q = pending[name]
                while q:
                    page = self._page_for(name, pending)
                    if page is None:
                        if id(q[0]) not in waited:
                            waited.add(id(q[0]))
                            self.stats["admissions_waited_for_memory"] += 1
                        break
                    page.submit([q.popleft() for _ in range(min(page.cap, len(q)))])
            if nxt < len(reqs) and all(p.busy is None for p in self.pages) and not any(pending.values()):
                # idle: sleep until the next arrival
                wait = reqs[nxt]["t"] - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.002))
        return done


class HostBatchPipeline:
    """Searches batches whose queries and results live in pinned host memory,
    with the copies overlapped: batch i's host-to-device copy runs on one copy
    stream while batch i - 1 searches, and batch i - 1's results come back on
    a second copy stream while batch i searches (two sets of device buffers
    alternate; events order every reuse).  Each batch is one kann_search_ex
    call with the given options; results equal those of that call."""

    def __init__(self, index, n, d, k, ef, device="cuda", **opts):
        self.index, self.n, self.k, self.ef, self.opts = index, n, k, ef, dict(opts)
        self.streams = [torch.cuda.Stream(device) for _ in range(3)]  # h2d, search, d2h
        self.q = [torch.empty((n, d), dtype=torch.float32, device=device) for _ in range(2)]
        self.ids = [torch.empty((n, k), dtype=torch.int32, device=device) for _ in range(2)]
        self.dists = [torch.empty((n, k), dtype=torch.float32, device=device) for _ in range(2)]
        ev = lambda: [torch.cuda.Event(), torch.cuda.Event()]
        self.ev_h2d, self.ev_search, self.ev_d2h = ev(), ev(), ev()
        self.i = 0

    def submit(self, q_host, ids_host, dists_host):
        """Queue batch q_host [n, d] (pinned FP32); its ids and distances land
        in ids_host / dists_host (pinned) once the d2h stream passes them."""
        hs, ss, ds = self.streams
        b = self.i & 1
        hs.wait_event(self.ev_search[b])  # the search two batches back has read q[b]
        with torch.cuda.stream(hs):
            self.q[b].copy_(q_host, non_blocking=True)
        self.ev_h2d[b].record(hs)
        ss.wait_event(self.ev_h2d[b])
        ss.wait_event(self.ev_d2h[b])  # the results two batches back have left ids[b]
        K.kann_search_ex(self.index, self.q[b], self.k, self.ef, ids=self.ids[b], dists=self.dists[b], stream=ss,
                         **self.opts)
        self.ev_search[b].record(ss)
        ds.wait_event(self.ev_search[b])
        with torch.cuda.stream(ds):
            ids_host.copy_(self.ids[b], non_blocking=True)
            dists_host.copy_(self.dists[b], non_blocking=True)
        self.ev_d2h[b].record(ds)
        self.i += 1

    def first_stream(self):
        return self.streams[0]

    def last_stream(self):
        return self.streams[2]

    def synchronize(self):
        for st in self.streams:
            st.synchronize()


def status_counts(done):
    """How many finished requests carry each KANN_QSTAT_* bit."""
    names = {"hop_cap": K.KANN_QSTAT_HOPCAP, "forgot": K.KANN_QSTAT_FORGOT, "bad_id": K.KANN_QSTAT_BAD_ID,
             "query_truncated": K.KANN_QSTAT_QUERY_TRUNCATED}
    return {n: int(sum(1 for r in done if r.get("status", 0) & b)) for n, b in names.items()}


def poisson_requests(rate, duration, index_queries, k_choices=(10, 100), ef_range=(64, 512), seed=0):
    """Poisson arrivals at `rate` per second for `duration` seconds; each
    request picks an index uniformly, a query of that index's query set, k
    uniformly from k_choices and ef uniformly from ef_range (inclusive)."""
    rng = np.random.default_rng(seed)
    names = list(index_queries)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            break
        name = names[rng.integers(len(names))]
        Q = index_queries[name]
        qi = int(rng.integers(len(Q)))
        out.append(dict(t=t, index=name, qid=qi, query=Q[qi], k=int(rng.choice(k_choices)),
                        ef=int(rng.integers(ef_range[0], ef_range[1] + 1))))
    return out


def latency_summary(done, duration):
    lat = np.array([r["latency"] for r in done]) * 1e3
    if len(lat) == 0:
        return {"completed": 0}
    return {"completed": len(done), "qps": len(done) / duration, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean())}
