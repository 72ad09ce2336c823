"""Per-index autotuner for the search launch settings.

The settings that do not change results — lanes per row gather, visited
table size, warps per CTA, plain vs persistent work-stealing launch — are
timed on a sample of the caller's queries with CUDA events; a setting is
accepted only if it returns exactly the same ids and distances as the
default launch (they all must: the search is defined by (k, ef) alone).
The winner is cached in a JSON file keyed by the index signature, the GPU
name and the driver version.
"""
import json
import os

import torch

from . import kann as K


def _signature(index, k, ef, rerank):
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    drv = torch.version.cuda or ""
    return "|".join(str(x) for x in (index.kind, index.dtype, index.d, index.n, index.M0, index.metric, k, ef,
                                      rerank, props.name, drv))


def _time(index, Q, k, ef, reps, opts):
    ctr = torch.zeros(1, dtype=torch.int32, device=Q.device) if opts.pop("persistent", False) else None
    run = lambda: K.kann_search_ex(index, Q, k, ef, work_counter=ctr, **opts)
    out = run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
    e0.record()
    for _ in range(reps):
        run()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, out


def tune(index, queries, k, ef, rerank=0, reps=5, cache_path=None, verbose=False):
    """Returns the fastest result-preserving option dict for kann_search_ex
    (keys lanes_per_row, hash_bits, warps_per_block, lean, persistent)."""
    key = _signature(index, k, ef, rerank)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            return dict(cache[key]["opts"])
    base_t, (ref_i, ref_d) = _time(index, queries, k, ef, reps, dict(rerank=rerank))
    best, best_t = dict(lanes_per_row=0, hash_bits=0, warps_per_block=0, lean=0, persistent=False), base_t
    results = []

    def trial(o):
        nonlocal best, best_t
        try:
            t, (ids, d) = _time(index, queries, k, ef, reps, dict(o, rerank=rerank))
        except K.KannError:
            return
        same = torch.equal(ids, ref_i) and torch.equal(d, ref_d)
        results.append((dict(o), t, same))
        if same and t < best_t:
            best, best_t = dict(o), t

    for lpr in (0, 2, 4, 8, 16, 32):
        for hb in (0, 9, 10, 11, 12):
            trial(dict(lanes_per_row=lpr, hash_bits=hb, warps_per_block=0, lean=0, persistent=False))
    for wpb in (1, 2, 4):
        for pers in (False, True):
            trial(dict(best, warps_per_block=wpb, persistent=pers))
    trial(dict(best, lean=1))
    if verbose:
        for o, t, same in sorted(results, key=lambda r: r[1])[:10]:
            print("%8.3f ms  same=%s  %s" % (t, same, o))
    if cache_path:
        cache[key] = {"opts": best, "ms": best_t, "default_ms": base_t}
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return dict(best)


def search_with(index, queries, k, ef, opts, rerank=0, **extra):
    """kann_search_ex with a tuned option dict (allocates the work counter
    for the persistent form)."""
    o = dict(opts)
    ctr = torch.zeros(1, dtype=torch.int32, device=queries.device) if o.pop("persistent", False) else None
    return K.kann_search_ex(index, queries, k, ef, rerank=rerank, work_counter=ctr, **o, **extra)
