"""Continuous-batching search server over resident indices.

Requests (index, query, k, ef) arrive over time.  The server keeps a fixed
set of batch slots per index, each with its own CUDA stream, device and
pinned host buffers and a CUDA graph of one persistent, work-stealing
`kann_search_batch` launch (mixed k and ef per query, the batch size read
from device memory so that one graph serves any batch up to the slot's
capacity).  Whenever a slot is free, the requests that have arrived and are
still waiting are admitted into it (up to its capacity) and launched; slots
run concurrently on their streams, so requests that arrive while earlier
batches are on the GPU start as soon as a slot frees up instead of waiting
for a global batch boundary.

Admission is by device memory: the slots are sized up front from a byte
budget (queries, per-query k/ef, outputs), and a request is admitted only
into a slot whose buffers it fits.  Every search step runs in the library's
kernels; this module only stages buffers, replays graphs and keeps time.
"""
import collections
import time

import numpy as np
import torch

from . import kann as K


class _Slot:
    def __init__(self, index, d, kmax, efmax, cap, device, opts):
        self.index, self.d, self.kmax, self.efmax, self.cap = index, d, kmax, efmax, cap
        self.stream = torch.cuda.Stream(device=device)
        f32, i32 = torch.float32, torch.int32
        self.q = torch.zeros((cap, d), dtype=f32, device=device)
        self.k = torch.ones(cap, dtype=i32, device=device)
        self.ef = torch.full((cap,), kmax, dtype=i32, device=device)
        self.n = torch.zeros(1, dtype=i32, device=device)
        self.counter = torch.zeros(1, dtype=i32, device=device)
        self.ids = torch.empty((cap, kmax), dtype=i32, device=device)
        self.dists = torch.empty((cap, kmax), dtype=f32, device=device)
        self.h_q = torch.zeros((cap, d), dtype=f32).pin_memory()
        self.h_k = torch.ones(cap, dtype=i32).pin_memory()
        self.h_ef = torch.full((cap,), kmax, dtype=i32).pin_memory()
        self.h_n = torch.zeros(1, dtype=i32).pin_memory()
        self.h_ids = torch.empty((cap, kmax), dtype=i32).pin_memory()
        self.h_dists = torch.empty((cap, kmax), dtype=f32).pin_memory()
        self.np_q, self.np_k, self.np_ef = self.h_q.numpy(), self.h_k.numpy(), self.h_ef.numpy()
        self.np_ids, self.np_dists = self.h_ids.numpy(), self.h_dists.numpy()
        self.opts = opts
        self.event = torch.cuda.Event()
        self.busy = None  # list of request records in flight
        self.graph = None

    def _launch(self):
        K.kann_search_batch(self.index, self.q, self.k, self.ef, kmax=self.kmax, efmax=self.efmax, ids=self.ids,
                            dists=self.dists, stream=self.stream, work_counter=self.counter, n_device=self.n,
                            **self.opts)

    def capture(self):
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

    def bytes(self):
        return K.kann_search_workspace_bytes(self.index, self.cap, self.kmax, self.efmax)

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
            self.event.record(self.stream)
        self.busy = reqs

    def poll(self):
        """Finished requests (with results filled in), or None if still running."""
        if self.busy is None or not self.event.query():
            return None
        reqs, self.busy = self.busy, None
        for i, r in enumerate(reqs):
            r["ids"] = self.np_ids[i, :r["k"]].copy()
            r["dists"] = self.np_dists[i, :r["k"]].copy()
        return reqs


class SearchServer:
    """indices: {name: dict(index=Index, d=..., kmax=..., efmax=...)}.
    memory_budget: device bytes for all slot buffers; slots_per_index and
    slot_capacity are reduced until the slots fit."""

    def __init__(self, indices, slots_per_index=3, slot_capacity=1024, memory_budget=1 << 30, device="cuda",
                 search_opts=None):
        self.slots = collections.OrderedDict()
        for name, spec in indices.items():
            cap = slot_capacity
            per = lambda c: K.kann_search_workspace_bytes(spec["index"], c, spec["kmax"], spec["efmax"])
            if per(cap) == 0:
                raise ValueError("index %r cannot run a search with kmax=%d efmax=%d" % (name, spec["kmax"],
                                                                                        spec["efmax"]))
            while cap > 16 and per(cap) * slots_per_index * len(indices) > memory_budget:
                cap //= 2
            self.slots[name] = [_Slot(spec["index"], spec["d"], spec["kmax"], spec["efmax"], cap, device,
                                      dict(search_opts or {}, **spec.get("opts", {})))
                                for _ in range(slots_per_index)]
        for ss in self.slots.values():
            for s in ss:
                s.capture()
        self.device_bytes = sum(s.bytes() for ss in self.slots.values() for s in ss)

    def run(self, requests, time_limit=None):
        """requests: list of dict(t=arrival seconds from start, index=name,
        query=float32[d], k=int, ef=int).  Serves them in arrival order,
        sleeping until each arrives; returns them with 'ids', 'dists',
        't_done' (seconds from start) and 'latency' (t_done - t)."""
        reqs = sorted(requests, key=lambda r: r["t"])
        pending = {name: collections.deque() for name in self.slots}
        nxt, done = 0, []
        t0 = time.perf_counter()
        while len(done) < len(reqs):
            now = time.perf_counter() - t0
            if time_limit is not None and now > time_limit:
                break
            while nxt < len(reqs) and reqs[nxt]["t"] <= now:
                pending[reqs[nxt]["index"]].append(reqs[nxt])
                nxt += 1
            for name, ss in self.slots.items():
                for s in ss:
                    fin = s.poll()
                    if fin is not None:
                        tnow = time.perf_counter() - t0
                        for r in fin:
                            r["t_done"] = tnow
                            r["latency"] = tnow - r["t"]
                        done.extend(fin)
                    if s.busy is None and pending[name]:
                        take = [pending[name].popleft() for _ in range(min(s.cap, len(pending[name])))]
                        s.submit(take)
            if nxt < len(reqs) and all(s.busy is None for ss in self.slots.values() for s in ss) and \
                    not any(pending.values()):
                # idle: sleep until the next arrival
                wait = reqs[nxt]["t"] - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.002))
        return done


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
