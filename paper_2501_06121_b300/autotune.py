"""Per-index autotuner for the search launch settings.

The settings that do not change results -- lanes per row gather, the
visited table's layout (compact 16-bit or wide 32-bit slots) and size,
warps per CTA, the team size (warps sharing one query), the lean register
budget, plain vs persistent work-stealing launch -- are timed on the caller's queries with CUDA events; a setting is
accepted only if it returns exactly the same ids and distances as the
default launch (they all must: the search is defined by (k, ef) alone).
The table size trades shared memory (hence queries resident per SM) against
forgotten ids that are evaluated again, and the best point moves with ef
and with the kernel's register budget, which is why it is measured rather
than fixed.  The winner is cached in a JSON file keyed by the index
signature, the GPU name and the driver version.
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


def tune(index, queries, k, ef, rerank=0, reps=5, cache_path=None, verbose=False, fixed=None):
    """Returns the fastest result-preserving option dict for kann_search_ex
    (keys lanes_per_row, hash_bits, visited_format, warps_per_block, lean,
    team, persistent).  `fixed`: options every trial runs with (such as a PQ
    table format), not tuned and not returned."""
    fixed = {key: v for key, v in (fixed or {}).items() if key not in ("rerank", "persistent")}
    key = _signature(index, k, ef, rerank) + "|" + json.dumps(fixed, sort_keys=True)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            return dict(cache[key]["opts"])
    base_t, (ref_i, ref_d) = _time(index, queries, k, ef, reps, dict(fixed, rerank=rerank))
    best = dict(lanes_per_row=0, hash_bits=0, visited_format=0, warps_per_block=0, lean=0, team=0,
                persistent=False)
    best_t = base_t
    results = []

    def trial(o):
        nonlocal best, best_t
        try:
            t, (ids, d) = _time(index, queries, k, ef, reps, dict(fixed, **o, rerank=rerank))
        except K.KannError:
            return
        same = torch.equal(ids, ref_i) and torch.equal(d, ref_d)
        results.append((dict(o), t, same))
        if same and t < best_t:
            best, best_t = dict(o), t

    tables = [(K.KANN_VISITED_COMPACT, hb) for hb in (11, 12, 13)] + [(K.KANN_VISITED_WIDE, hb) for hb in (10, 11)]
    for vf, hb in tables:
        trial(dict(best, visited_format=vf, hash_bits=hb))
    for lpr in (2, 4, 8, 16, 32):
        trial(dict(best, lanes_per_row=lpr))
    for wpb in (1, 2, 4):
        for pers in (False, True):
            trial(dict(best, warps_per_block=wpb, persistent=pers))
    trial(dict(best, lean=1))
    # teams of 2 and 4 warps per query: more warps per SM when each query's
    # shared memory (beam, visited table) is what limits them
    for team in (2, 4):
        for pers in (False, True):
            trial(dict(best, team=team, warps_per_block=0, lean=0, persistent=pers))
    # the table size again, at the chosen lane mapping and CTA shape
    for vf, hb in tables:
        trial(dict(best, visited_format=vf, hash_bits=hb))
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
