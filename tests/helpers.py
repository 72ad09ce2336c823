"""Shared test helpers: graph invariants, golden fixtures, comparisons."""
import json
import os
from collections import deque

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def golden_graph(case):
    """Serialised graph dict (see include/kann.h) from a hand-written case."""
    n = len(case["x"])
    M, M0, L = case["M"], case["M0"], case["max_level"]
    level = np.array(case["level"], np.int8)
    l0 = np.array(case["l0"], np.int32)
    slot = np.full(n, -1, np.int32)
    ups = sorted(int(k) for k in case["upper"])
    upper = np.full((max(len(ups), 1), max(L, 1), M), -1, np.int32)
    for s, v in enumerate(ups):
        slot[v] = s
        for li, row in enumerate(case["upper"][str(v)]):
            upper[s, li, :len(row)] = row
    return dict(n=n, M=M, M0=M0, max_level=L, entry=case["entry"], level=level, l0=l0, upper_slot=slot,
                upper=upper)


def layer_lists(g, v, layer):
    if layer == 0:
        row = g["l0"][v]
    else:
        row = g["upper"][g["upper_slot"][v], layer - 1]
    return [int(u) for u in row if u >= 0]


def graph_problems(g, max_unreachable=0.01):
    """Every violated HNSW invariant (empty list = all hold): degree caps,
    no self loops, no duplicate edges, ids in range, edges only between
    nodes present on the layer, upper slots consistent with levels, entry
    point of maximum level, at least one out-edge per node of a layer with
    more than one node, and at most `max_unreachable` of a layer's nodes
    unreachable from the entry point within the layer.  (Insertion with
    heuristic pruning of back-links does not guarantee full reachability:
    a node whose every in-edge was pruned away keeps its out-edges only.)"""
    n, M, M0, L = g["n"], g["M"], g["M0"], g["max_level"]
    level = g["level"].astype(int)
    out = []
    if M0 != 2 * M:
        out.append("M0 != 2M")
    if level.max() != L:
        out.append("max_level is not the largest level")
    if level[g["entry"]] != L:
        out.append("entry point is not on the top layer")
    us = g["upper_slot"]
    if not np.all((level >= 1) == (us >= 0)):
        out.append("upper slot present exactly for level >= 1 violated")
    for layer in range(L + 1):
        nodes = np.nonzero(level >= layer)[0]
        present = level >= layer
        cap = M0 if layer == 0 else M
        adj = {}
        for v in nodes:
            lst = layer_lists(g, v, layer)
            if len(lst) > cap:
                out.append("degree cap at layer %d node %d" % (layer, v))
            if len(lst) == 0 and len(nodes) > 1:
                out.append("node %d has no out-edge at layer %d" % (v, layer))
            if v in lst:
                out.append("self loop %d at layer %d" % (v, layer))
            if len(set(lst)) != len(lst):
                out.append("duplicate edge at node %d layer %d" % (v, layer))
            for u in lst:
                if not (0 <= u < n) or not present[u]:
                    out.append("edge %d->%d at layer %d leaves the layer" % (v, u, layer))
            adj[int(v)] = lst
        seen = {int(g["entry"])}
        dq = deque([int(g["entry"])])
        while dq:
            v = dq.popleft()
            for u in adj.get(v, []):
                if u not in seen:
                    seen.add(u)
                    dq.append(u)
        if len(nodes) - len(seen) > max_unreachable * len(nodes):
            out.append("layer %d: %d of %d nodes unreachable" % (layer, len(nodes) - len(seen), len(nodes)))
        if len(out) > 20:
            break
    return out


def recall(ids, gt_ids, k):
    return float(np.mean([len(set(a[:k]) & set(b[:k])) / k for a, b in zip(ids, gt_ids)]))


def id_set_match_fraction(a, b):
    return float(np.mean([set(x) == set(y) for x, y in zip(a, b)]))


def random_graph(n, M, levels, seed):
    """A seeded random HNSW-shaped graph over n nodes (an input, like the
    data: search parity holds on any graph, navigable or not): the given
    levels, layer-0 lists of 2M distinct random other nodes, and for every
    layer l >= 1 lists of min(M, nodes on l - 1) distinct random other nodes
    of that layer; the entry point is the lowest id on the top layer."""
    rng = np.random.default_rng(seed)
    M0 = 2 * M
    levels = np.asarray(levels, np.int8)
    L = int(levels.max()) if n else 0

    def rows(cands):
        # for each node of cands, min(M, |cands| - 1) distinct other nodes of cands
        m = min(M, len(cands) - 1)
        out = np.empty((len(cands), m), np.int64)
        for i in range(len(cands)):
            pick = rng.choice(len(cands) - 1, m, replace=False)
            out[i] = pick + (pick >= i)  # skip position i (the node itself)
        return cands[out]

    l0 = np.full((n, M0), -1, np.int32)
    m0 = min(M0, n - 1)
    if m0 * m0 > n // 8:
        # small n: distinct draws per row
        picks = np.stack([rng.choice(n - 1, m0, replace=False) for _ in range(n)]) if n > 1 else \
            np.zeros((n, 0), np.int64)
    else:
        # large n: independent draws, the few rows with a repeat drawn again
        # (a row repeats with probability below 1/16 here)
        picks = rng.integers(0, n - 1, (n, m0))
        while True:
            srt = np.sort(picks, axis=1)
            bad = np.nonzero((srt[:, 1:] == srt[:, :-1]).any(axis=1))[0]
            if len(bad) == 0:
                break
            picks[bad] = rng.integers(0, n - 1, (len(bad), m0))
    picks = picks + (picks >= np.arange(n)[:, None])
    l0[:, :m0] = picks
    upper_nodes = np.nonzero(levels >= 1)[0]
    slot = np.full(n, -1, np.int32)
    slot[upper_nodes] = np.arange(len(upper_nodes), dtype=np.int32)
    upper = np.full((max(len(upper_nodes), 1), max(L, 1), M), -1, np.int32)
    for layer in range(1, L + 1):
        on = np.nonzero(levels >= layer)[0]
        if len(on) < 2:
            continue
        r = rows(on)
        upper[slot[on], layer - 1, :r.shape[1]] = r
    entry = int(np.nonzero(levels == L)[0][0])
    return dict(n=n, M=M, M0=M0, max_level=L, entry=entry, level=levels, l0=l0, upper_slot=slot, upper=upper)
