"""Autotuner of the batched sweeps: chooses the work-item order, the column
groups per work item, the persistent grid size and the tile height of the
constrained-transport sweeps (rows of columns per work-item group) of a
fish_batch by timing whole double steps of a scratch batch with the same
boxes, and caches the choice per batch geometry and GPU in a JSON file next
to the built library.  The schedule (order, groups, grid) is searched at
the default tile height first, then every tile height with the best
schedule.

The tuned parameters change only the scheduling of the work (which block
marches which columns when), never the arithmetic, so every choice gives the
same result.
"""
from __future__ import annotations

import hashlib
import itertools
import json
import os

from . import (FISH_BATCH_OPT_CTROWS, FISH_BATCH_OPT_GRID, FISH_BATCH_OPT_GROUPS, FISH_BATCH_OPT_ORDER, Batch)

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")
ORDERS = (0, 1, 2)
GROUPS = (1, 2, 4)
GRIDS = (1, 2)
CTROWS = (4, 8)


def signature(dims, gammas, bcs, device_name):
    text = json.dumps([list(map(list, dims)), list(gammas), list(bcs), device_name])
    return hashlib.sha1(text.encode()).hexdigest()


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except Exception:
        return {}


def _save(db):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + ".%d.tmp" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(db, f, indent=1)
    os.replace(tmp, CACHE)


def apply(batch, choice):
    batch.set_option(FISH_BATCH_OPT_ORDER, choice["order"])
    batch.set_option(FISH_BATCH_OPT_GROUPS, choice["groups"])
    batch.set_option(FISH_BATCH_OPT_GRID, choice["grid"])
    batch.set_option(FISH_BATCH_OPT_CTROWS, choice.get("ctrows", 4))


def tune(dims, gammas, bcs, states, hs=None, k=0.5, steps=2, use_cache=True, candidates=None):
    """Best {"order", "groups", "grid", "ms"} for a batch of these boxes
    (``states``: initial state of every box), timed on the current GPU."""
    import torch
    dev = torch.cuda.get_device_name()
    key = signature(dims, gammas, bcs, dev)
    db = _load() if use_cache else {}
    if use_cache and key in db:
        return db[key]
    cands = candidates or [dict(order=o, groups=g, grid=r, ctrows=CTROWS[0])
                           for o, g, r in itertools.product(ORDERS, GROUPS, GRIDS)]
    b = Batch(dims, gammas, bcs, hs)

    def timed(c):
        apply(b, c)
        for i, st in enumerate(states):
            b.set_state(i, st)
        b.step(k, 1)  # capture and warm
        b.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(b.stream)
        b.step(k, steps)
        e1.record(b.stream)
        e1.synchronize()
        b.sync()
        return e0.elapsed_time(e1) / steps

    try:
        results = [(timed(c), c) for c in cands]
        if candidates is None:
            # second stage: the other tile heights with the best schedule
            _, best = min(results, key=lambda x: x[0])
            for rows in CTROWS[1:]:
                c = dict(best, ctrows=rows)
                results.append((timed(c), c))
        ms, best = min(results, key=lambda x: x[0])
        choice = dict(best, ms=ms, tried=[dict(c, ms=t) for t, c in results])
    finally:
        b.close()
    if use_cache:
        db[key] = choice
        _save(db)
    return choice
